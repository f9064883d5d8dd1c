// C-ABI entry points of libhmfsr: host-side validation, workspace layout and launches.
#include <math.h>
#include <string.h>

#include "hmfsr_internal.cuh"

using namespace hmfsr;

#ifdef HMFSR_CHECKED
// the checked build's error word: 0, or the source line of the first access that lay
// outside every buffer of its call
__device__ int g_check_err;
#endif

namespace {

// the buffers of the entry-point call running on this host thread (checked build)
thread_local CheckRanges t_check = {};
#ifdef HMFSR_CHECKED
size_t g_check_shrink = 0;  // test hook of the checked build: bytes taken off each registered workspace
#endif

// For the duration of one entry-point call: the caller's buffers, as its kernels may read
// and write them (checked build; nothing in the default build).
struct CheckScope {
#ifdef HMFSR_CHECKED
    CheckScope() {
        t_check = CheckRanges{};
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_check_err) == cudaSuccess) t_check.err = static_cast<int *>(p);
        else cudaGetLastError();
    }
    ~CheckScope() { t_check = CheckRanges{}; }
    void add(const void *p, size_t bytes) {
        if (!p || t_check.n >= kCheckMaxRanges) return;
        t_check.lo[t_check.n] = static_cast<const char *>(p);
        t_check.hi[t_check.n] = static_cast<const char *>(p) + bytes;
        ++t_check.n;
    }
    void add_ws(const void *p, size_t bytes) { add(p, bytes > g_check_shrink ? bytes - g_check_shrink : 0); }
#else
    void add(const void *, size_t) {}
    void add_ws(const void *, size_t) {}
#endif
};

// bytes of a burst as the kernels may read it: frames h x pitch apart, the last row of
// the last frame `width` samples long
size_t burst_bytes(const hmfsr_burst_desc *d) {
    return (((size_t)d->n_frames - 1) * d->height + d->height - 1) * d->pitch_elems * 2 + (size_t)d->width * 2;
}
size_t motion_bytes(const Geom &g) { return (size_t)g.n * g.ty * g.tx * 2 * sizeof(float); }
size_t rgb_bytes(const hmfsr_burst_desc *d, int num, int den) {
    return 3 * (size_t)(((long long)d->height * num) / den) * (size_t)(((long long)d->width * num) / den) * sizeof(float);
}

constexpr size_t kAlign = 256;
inline size_t align_up(size_t x) { return (x + kAlign - 1) & ~(kAlign - 1); }

// Bump allocator over the caller's workspace (or a null base for size queries).
struct Carver {
    char *base;
    size_t off = 0;
    explicit Carver(void *b) : base(static_cast<char *>(b)) {}
    template <typename T>
    T *take(size_t count) {
        size_t o = off;
        off = align_up(off + count * sizeof(T));
        return base ? reinterpret_cast<T *>(base + o) : nullptr;
    }
};

bool valid_desc(const hmfsr_burst_desc *d, hmfsr_status *why) {
    *why = HMFSR_ERR_INVALID_ARG;
    if (!d) return false;
    if (d->n_frames < 1 || d->n_frames > 4096) return false;
    if (d->height < 4 || d->width < 4 || (d->height & 1) || (d->width & 1)) return false;
    // at most 65536 x 65536: a half-res plane stays below 2^31 texels (32-bit offsets)
    if (d->height > 65536 || d->width > 65536) return false;
    if (d->pitch_elems < d->width || (d->pitch_elems & 1)) return false;
    // one frame holds fewer than 2^31 samples (32-bit offsets within a frame)
    if ((long long)d->height * d->pitch_elems >= (1LL << 31)) return false;
    if (d->ref < 0 || d->ref >= d->n_frames) return false;
    // 3x3 sums of a 16-bit guide channel must fit 16 bits, Lq 16 bits
    if (d->white_level < 1 || d->white_level > 7281) return false;
    if (d->cfa != 0 || d->black_level != 0) { *why = HMFSR_ERR_UNSUPPORTED; return false; }
    return true;
}

bool valid_tile(int tile) { return tile == 8 || tile == 16 || tile == 32 || tile == 64; }

bool valid_scale(int num, int den) { return num >= 1 && den >= 1 && num <= 8 && den <= 8 && num >= den && num <= 4 * den; }

bool finite_pos(float x) { return isfinite(x) && x > 0.f; }
bool finite_nonneg(float x) { return isfinite(x) && x >= 0.f; }

bool valid_merge_params(const hmfsr_merge_params *p) {
    if (!p) return false;
    if (!finite_pos(p->k_detail) || !finite_pos(p->k_denoise) || !finite_pos(p->d_tr) || !finite_pos(p->k_stretch) ||
        !finite_pos(p->k_shrink))
        return false;
    if (!isfinite(p->d_th) || !isfinite(p->t) || !finite_nonneg(p->s1) || !finite_nonneg(p->s2) || !isfinite(p->m_th))
        return false;
    if (!finite_nonneg(p->noise_a) || !finite_nonneg(p->noise_b)) return false;
    return valid_tile(p->tile);
}

bool valid_align_params(const hmfsr_align_params *p) {
    if (!p || !valid_tile(p->tile) || p->n_levels < 1 || p->n_levels > 4 || p->lk_iters < 0 || p->lk_iters > 16)
        return false;
    for (int l = 0; l < 4; ++l)
        if (p->radius[l] < 0 || p->radius[l] > 7) return false;
    return true;
}

Geom make_geom(const hmfsr_burst_desc *d, int tile) {
    Geom g;
    g.n = d->n_frames; g.h = d->height; g.w = d->width; g.pitch = d->pitch_elems; g.ref = d->ref;
    g.wl = d->white_level; g.hh = d->height / 2; g.wh = d->width / 2;
    g.tile = tile; g.ty = div_up(d->height, tile); g.tx = div_up(d->width, tile);
    return g;
}

// alignment workspace: pyramid levels and the integer vectors of every level
size_t carve_align(void *ws, const Geom &g, int tile, int n_levels_max, AlignLevels *L) {
    static const int fac[3] = {2, 4, 4};
    Carver c(ws);
    int t = tile / 2;
    L->lh[0] = g.hh; L->lw[0] = g.wh;
    int nl = 1;
    while (nl < n_levels_max && nl < 4) {
        int nh = L->lh[nl - 1] / fac[nl - 1], nw = L->lw[nl - 1] / fac[nl - 1];
        if (nh < 16 || nw < 16) break;
        L->lh[nl] = nh; L->lw[nl] = nw;
        ++nl;
    }
    L->n_levels = nl;
    for (int l = 0; l < nl; ++l) {
        L->lty[l] = div_up(L->lh[l], t);
        L->ltx[l] = div_up(L->lw[l], t);
        L->img[l] = c.take<uint16_t>((size_t)g.n * L->lh[l] * L->lw[l]);
        L->vec[l] = c.take<int2>((size_t)g.n * L->lty[l] * L->ltx[l]);
    }
    return c.off;
}

size_t carve_merge(void *ws, const Geom &g, MergePlanes *P) {
    Carver c(ws);
    size_t hw = (size_t)g.hh * g.wh;
    P->s1 = c.take<uint2>(g.n * hw);
    P->base_stats = c.take<float4>(hw);
    P->kern = c.take<float4>(g.n * hw);
    P->rhat = c.take<float>(g.n * hw);
    P->s_tile = c.take<float>((size_t)g.n * g.ty * g.tx);
    P->geo = c.take<int4>((size_t)g.n * g.ty * g.tx);
    P->hf_flag = c.take<unsigned char>(hw);
    return c.off;
}

// Bounded-memory merge workspace: a sub-burst of slots = min(n, chunk + 1) packed frames
// (slot 0 the base frame), their motion rows, the merge planes of that sub-burst, and the
// running sums of every output pixel (9 planes of Ho x Wo floats).
struct ChunkLayout {
    uint16_t *sub = nullptr;
    float *sub_motion = nullptr;
    MergePlanes P;
    float *state = nullptr;
    hmfsr_burst_desc sd;
    Geom gs;
};

size_t carve_chunked(void *ws, const hmfsr_burst_desc *d, int tile, int num, int den, int chunk, ChunkLayout *L) {
    L->sd = *d;
    L->sd.n_frames = d->n_frames < chunk + 1 ? d->n_frames : chunk + 1;
    L->sd.pitch_elems = d->width;
    L->sd.ref = 0;
    L->gs = make_geom(&L->sd, tile);
    const size_t ho = (size_t)(((long long)d->height * num) / den), wo = (size_t)(((long long)d->width * num) / den);
    Carver c(ws);
    L->sub = c.take<uint16_t>((size_t)L->sd.n_frames * d->height * d->width);
    L->sub_motion = c.take<float>((size_t)L->sd.n_frames * L->gs.ty * L->gs.tx * 2);
    const size_t planes = carve_merge(ws ? static_cast<char *>(ws) + c.off : nullptr, L->gs, &L->P);
    c.off = align_up(c.off + planes);
    L->state = c.take<float>(9 * ho * wo);
    return c.off;
}

MergeConsts consts_of(const hmfsr_merge_params *p) {
    MergeConsts c;
    c.k_detail = p->k_detail; c.k_denoise = p->k_denoise; c.d_th = p->d_th; c.d_tr = p->d_tr;
    c.k_stretch = p->k_stretch; c.k_shrink = p->k_shrink; c.t = p->t; c.s1 = p->s1; c.s2 = p->s2;
    c.m_th = p->m_th; c.noise_a = p->noise_a; c.noise_b = p->noise_b;
    c.noise_table = nullptr;
    c.hf_loss = 0.f;
    return c;
}

hmfsr_status check_ws(void *ws, size_t ws_bytes, size_t need) {
    if (need == 0) return HMFSR_OK;
    if (!ws || ws_bytes < need || (reinterpret_cast<uintptr_t>(ws) & (kAlign - 1))) return HMFSR_ERR_WORKSPACE;
    return HMFSR_OK;
}

bool aligned4(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 3) == 0; }
bool aligned8(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 7) == 0; }

hmfsr_status cuda_status(cudaError_t e) { return e == cudaSuccess ? HMFSR_OK : HMFSR_ERR_CUDA; }

// The calling host thread's side stream on one device (highest priority) and the two
// events that fork it from, and join it back to, the caller's stream.
struct SideStream {
    cudaStream_t s = nullptr;
    cudaEvent_t fork = nullptr, join = nullptr, aux = nullptr;
    ~SideStream() {
        if (fork) cudaEventDestroy(fork);
        if (join) cudaEventDestroy(join);
        if (aux) cudaEventDestroy(aux);
        if (s) cudaStreamDestroy(s);
    }
};
constexpr int kMaxSideDevices = 64;
thread_local SideStream t_side[kMaxSideDevices];

// nullptr when the device has none and one cannot be made
SideStream *side_stream() {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxSideDevices) return nullptr;
    SideStream &ss = t_side[dev];
    if (ss.s) return &ss;
    int least = 0, greatest = 0;
    if (cudaDeviceGetStreamPriorityRange(&least, &greatest) != cudaSuccess) return nullptr;
    cudaStream_t s = nullptr;
    cudaEvent_t a = nullptr, b = nullptr, x = nullptr;
    if (cudaStreamCreateWithPriority(&s, cudaStreamNonBlocking, greatest) != cudaSuccess ||
        cudaEventCreateWithFlags(&a, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&b, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&x, cudaEventDisableTiming) != cudaSuccess) {
        if (a) cudaEventDestroy(a);
        if (b) cudaEventDestroy(b);
        if (s) cudaStreamDestroy(s);
        return nullptr;
    }
    ss.s = s;
    ss.fork = a;
    ss.join = b;
    ss.aux = x;
    return &ss;
}

}  // namespace

const CheckRanges &hmfsr::current_check_ranges() { return t_check; }

extern "C" {

size_t hmfsr_workspace_size(int op, const hmfsr_burst_desc *desc, int tile, int scale_num, int scale_den) {
    hmfsr_status why;
    if (!valid_desc(desc, &why) || !valid_tile(tile)) return 0;
    Geom g = make_geom(desc, tile);
    if (op == HMFSR_OP_ALIGN) {
        AlignLevels L;
        return carve_align(nullptr, g, tile, 4, &L);
    }
    if (op == HMFSR_OP_MERGE || op == HMFSR_OP_MERGE_STAGES) {
        if (op == HMFSR_OP_MERGE && !valid_scale(scale_num, scale_den)) return 0;
        MergePlanes P;
        return carve_merge(nullptr, g, &P);
    }
    if (op == HMFSR_OP_ALIGN_MERGE) {
        if (!valid_scale(scale_num, scale_den)) return 0;
        AlignLevels L;
        MergePlanes P;
        return carve_align(nullptr, g, tile, 4, &L) + carve_merge(nullptr, g, &P);
    }
    if (op == HMFSR_OP_MERGE_BACKWARD) {
        if (!valid_scale(scale_num, scale_den)) return 0;
        MergePlanes P;
        BwdPlanes B;
        const int ho = (int)(((long long)desc->height * scale_num) / scale_den);
        const int wo = (int)(((long long)desc->width * scale_num) / scale_den);
        return carve_backward(nullptr, g, ho, wo, carve_merge(nullptr, g, &P), &B);
    }
    return 0;
}

hmfsr_status hmfsr_align(const uint16_t *burst_dev, const hmfsr_burst_desc *desc, const hmfsr_align_params *params,
                         float *motion_dev, int32_t *motion_int_dev, void *ws, size_t ws_bytes, void *stream) {
    hmfsr_status why;
    if (!valid_desc(desc, &why)) return why;
    if (!burst_dev || !motion_dev || !aligned4(burst_dev) || !valid_align_params(params)) return HMFSR_ERR_INVALID_ARG;
    Geom g = make_geom(desc, params->tile);
    AlignLevels L;
    size_t need = carve_align(nullptr, g, params->tile, params->n_levels, &L);
    hmfsr_status st = check_ws(ws, ws_bytes, need);
    if (st != HMFSR_OK) return st;
    carve_align(ws, g, params->tile, params->n_levels, &L);
    CheckScope chk;
    chk.add(burst_dev, burst_bytes(desc));
    chk.add(motion_dev, motion_bytes(g));
    chk.add(motion_int_dev, motion_bytes(g));
    chk.add_ws(ws, need);
    return cuda_status(launch_align(burst_dev, g, *params, L, motion_dev, motion_int_dev, (cudaStream_t)stream));
}

hmfsr_status hmfsr_align_quadfit(const uint16_t *burst_dev, const hmfsr_burst_desc *desc,
                                 const hmfsr_align_params *params, float *motion_dev, int32_t *motion_int_dev,
                                 void *ws, size_t ws_bytes, void *stream) {
    hmfsr_status why;
    if (!valid_desc(desc, &why)) return why;
    if (!burst_dev || !motion_dev || !aligned4(burst_dev) || !valid_align_params(params)) return HMFSR_ERR_INVALID_ARG;
    Geom g = make_geom(desc, params->tile);
    AlignLevels L;
    size_t need = carve_align(nullptr, g, params->tile, params->n_levels, &L);
    hmfsr_status st = check_ws(ws, ws_bytes, need);
    if (st != HMFSR_OK) return st;
    carve_align(ws, g, params->tile, params->n_levels, &L);
    CheckScope chk;
    chk.add(burst_dev, burst_bytes(desc));
    chk.add(motion_dev, motion_bytes(g));
    chk.add(motion_int_dev, motion_bytes(g));
    chk.add_ws(ws, need);
    return cuda_status(launch_align_quadfit(burst_dev, g, *params, L, motion_dev, motion_int_dev,
                                            (cudaStream_t)stream));
}

hmfsr_status hmfsr_merge(const uint16_t *burst_dev, const hmfsr_burst_desc *desc, const float *motion_dev,
                         const hmfsr_merge_params *params, int scale_num, int scale_den, float *rgb_dev,
                         float *den_dev, void *ws, size_t ws_bytes, void *stream) {
    hmfsr_status why;
    if (!valid_desc(desc, &why)) return why;
    if (!burst_dev || !motion_dev || !rgb_dev || !aligned4(burst_dev) || !aligned8(motion_dev) || !valid_merge_params(params) ||
        !valid_scale(scale_num, scale_den))
        return HMFSR_ERR_INVALID_ARG;
    Geom g = make_geom(desc, params->tile);
    MergePlanes P;
    size_t need = carve_merge(nullptr, g, &P);
    hmfsr_status st = check_ws(ws, ws_bytes, need);
    if (st != HMFSR_OK) return st;
    carve_merge(ws, g, &P);
    cudaStream_t s = (cudaStream_t)stream;
    MergeConsts c = consts_of(params);
    CheckScope chk;
    chk.add(burst_dev, burst_bytes(desc));
    chk.add(motion_dev, motion_bytes(g));
    chk.add(rgb_dev, rgb_bytes(desc, scale_num, scale_den));
    chk.add(den_dev, rgb_bytes(desc, scale_num, scale_den));
    chk.add_ws(ws, need);
    cudaError_t e = launch_merge_prep(burst_dev, motion_dev, g, c, P, s);
    if (e != cudaSuccess) return HMFSR_ERR_CUDA;
    return cuda_status(launch_merge_accum(burst_dev, motion_dev, g, P, scale_num, scale_den, rgb_dev, den_dev, s));
}

hmfsr_status hmfsr_align_merge(const uint16_t *burst_dev, const hmfsr_burst_desc *desc,
                               const hmfsr_align_params *aparams, const hmfsr_merge_params *mparams, int scale_num,
                               int scale_den, float *motion_dev, int32_t *motion_int_dev, float *rgb_dev,
                               float *den_dev, void *ws, size_t ws_bytes, void *stream) {
    hmfsr_status why;
    if (!valid_desc(desc, &why)) return why;
    if (!burst_dev || !motion_dev || !rgb_dev || !aligned4(burst_dev) || !aligned8(motion_dev) ||
        !valid_align_params(aparams) || !valid_merge_params(mparams) || aparams->tile != mparams->tile ||
        !valid_scale(scale_num, scale_den))
        return HMFSR_ERR_INVALID_ARG;
    Geom g = make_geom(desc, mparams->tile);
    AlignLevels L;
    MergePlanes P;
    const size_t align_bytes = carve_align(nullptr, g, aparams->tile, 4, &L);
    const size_t need = align_bytes + carve_merge(nullptr, g, &P);
    hmfsr_status st = check_ws(ws, ws_bytes, need);
    if (st != HMFSR_OK) return st;
    carve_align(ws, g, aparams->tile, aparams->n_levels, &L);
    carve_merge(static_cast<char *>(ws) + align_bytes, g, &P);
    SideStream *side = side_stream();
    if (!side) return HMFSR_ERR_CUDA;
    cudaStream_t s = (cudaStream_t)stream;
    const MergeConsts c = consts_of(mparams);
    CheckScope chk;
    chk.add(burst_dev, burst_bytes(desc));
    chk.add(motion_dev, motion_bytes(g));
    chk.add(motion_int_dev, motion_bytes(g));
    chk.add(rgb_dev, rgb_bytes(desc, scale_num, scale_den));
    chk.add(den_dev, rgb_bytes(desc, scale_num, scale_den));
    chk.add_ws(ws, need);
    // fork: the alignment on the side stream, the motion-free preparation here
    if (cudaEventRecord(side->fork, s) != cudaSuccess || cudaStreamWaitEvent(side->s, side->fork, 0) != cudaSuccess)
        return HMFSR_ERR_CUDA;
    const cudaError_t ea = launch_align(burst_dev, g, *aparams, L, motion_dev, motion_int_dev, side->s);
    // the join is recorded even after a failed launch, so the side stream never runs ahead
    // of a later fork unordered
    const cudaError_t ej = cudaEventRecord(side->join, side->s);
    const cudaError_t ef = launch_merge_prep_frames(burst_dev, g, c, P, s);
    const cudaError_t ew = cudaStreamWaitEvent(s, side->join, 0);
    if (ea != cudaSuccess || ej != cudaSuccess || ef != cudaSuccess || ew != cudaSuccess) return HMFSR_ERR_CUDA;
    if (launch_merge_prep_motion(motion_dev, g, c, P, s) != cudaSuccess) return HMFSR_ERR_CUDA;
    return cuda_status(launch_merge_accum(burst_dev, motion_dev, g, P, scale_num, scale_den, rgb_dev, den_dev, s));
}

size_t hmfsr_merge_chunked_workspace_size(const hmfsr_burst_desc *desc, int tile, int scale_num, int scale_den,
                                          int chunk_frames) {
    hmfsr_status why;
    if (!valid_desc(desc, &why) || !valid_tile(tile) || !valid_scale(scale_num, scale_den) || chunk_frames < 1 ||
        chunk_frames > 4096)
        return 0;
    ChunkLayout L;
    return carve_chunked(nullptr, desc, tile, scale_num, scale_den, chunk_frames, &L);
}

hmfsr_status hmfsr_merge_chunked(const uint16_t *burst_dev, const hmfsr_burst_desc *desc, const float *motion_dev,
                                 const hmfsr_merge_params *params, int scale_num, int scale_den, int chunk_frames,
                                 float *rgb_dev, float *den_dev, void *ws, size_t ws_bytes, void *stream) {
    hmfsr_status why;
    if (!valid_desc(desc, &why)) return why;
    if (!burst_dev || !motion_dev || !rgb_dev || !aligned4(burst_dev) || !aligned8(motion_dev) ||
        !valid_merge_params(params) || !valid_scale(scale_num, scale_den) || chunk_frames < 1 || chunk_frames > 4096)
        return HMFSR_ERR_INVALID_ARG;
    ChunkLayout L;
    const size_t need = carve_chunked(nullptr, desc, params->tile, scale_num, scale_den, chunk_frames, &L);
    hmfsr_status st = check_ws(ws, ws_bytes, need);
    if (st != HMFSR_OK) return st;
    carve_chunked(ws, desc, params->tile, scale_num, scale_den, chunk_frames, &L);
    const Geom g = make_geom(desc, params->tile);
    cudaStream_t s = (cudaStream_t)stream;
    const MergeConsts c = consts_of(params);
    CheckScope chk;
    chk.add(burst_dev, burst_bytes(desc));
    chk.add(motion_dev, motion_bytes(g));
    chk.add(rgb_dev, rgb_bytes(desc, scale_num, scale_den));
    chk.add(den_dev, rgb_bytes(desc, scale_num, scale_den));
    chk.add_ws(ws, need);
    const size_t frame_px = (size_t)desc->height * desc->width, motion_row = (size_t)g.ty * g.tx * 2;
    // one frame of the burst into a slot of the packed sub-burst, with its motion row
    auto put = [&](int f, int slot) -> bool {
        const uint16_t *src = burst_dev + (size_t)f * desc->height * desc->pitch_elems;
        if (cudaMemcpy2DAsync(L.sub + (size_t)slot * frame_px, (size_t)desc->width * 2, src,
                              (size_t)desc->pitch_elems * 2, (size_t)desc->width * 2, desc->height,
                              cudaMemcpyDeviceToDevice, s) != cudaSuccess)
            return false;
        return cudaMemcpyAsync(L.sub_motion + (size_t)slot * motion_row, motion_dev + (size_t)f * motion_row,
                               motion_row * sizeof(float), cudaMemcpyDeviceToDevice, s) == cudaSuccess;
    };
    if (!put(desc->ref, 0)) return HMFSR_ERR_CUDA;
    const int others = desc->n_frames - 1;
    const int chunks = others > 0 ? (others + chunk_frames - 1) / chunk_frames : 1;
    for (int ci = 0; ci < chunks; ++ci) {
        const int o0 = ci * chunk_frames;
        const int m = others - o0 < chunk_frames ? others - o0 : chunk_frames;
        for (int j = 0; j < m; ++j) {
            const int o = o0 + j, f = o < desc->ref ? o : o + 1;  // the others in order
            if (!put(f, 1 + j)) return HMFSR_ERR_CUDA;
        }
        Geom gc = L.gs;
        gc.n = 1 + (m > 0 ? m : 0);
        // the base frame's planes (slot 0) are made by the first chunk and kept
        if (launch_merge_prep_frames(L.sub, gc, c, L.P, s, ci > 0 ? 1 : 0) != cudaSuccess ||
            launch_merge_prep_motion(L.sub_motion, gc, c, L.P, s) != cudaSuccess)
            return HMFSR_ERR_CUDA;
        const bool last = (ci == chunks - 1);
        if (launch_merge_accum_chunk(L.sub, L.sub_motion, gc, L.P, scale_num, scale_den, rgb_dev, den_dev,
                                     ci > 0 ? L.state : nullptr, last ? nullptr : L.state, ci > 0, s) != cudaSuccess)
            return HMFSR_ERR_CUDA;
    }
    return HMFSR_OK;
}

hmfsr_status hmfsr_merge_noise(const uint16_t *burst_dev, const hmfsr_burst_desc *desc, const float *motion_dev,
                               const hmfsr_merge_params *params, const float *noise_table_dev, int scale_num,
                               int scale_den, float *rgb_dev, float *den_dev, void *ws, size_t ws_bytes,
                               void *stream) {
    hmfsr_status why;
    if (!valid_desc(desc, &why)) return why;
    if (!noise_table_dev || (reinterpret_cast<uintptr_t>(noise_table_dev) & 15)) return HMFSR_ERR_INVALID_ARG;
    if (!burst_dev || !motion_dev || !rgb_dev || !aligned4(burst_dev) || !aligned8(motion_dev) || !valid_merge_params(params) ||
        !valid_scale(scale_num, scale_den))
        return HMFSR_ERR_INVALID_ARG;
    Geom g = make_geom(desc, params->tile);
    MergePlanes P;
    size_t need = carve_merge(nullptr, g, &P);
    hmfsr_status st = check_ws(ws, ws_bytes, need);
    if (st != HMFSR_OK) return st;
    carve_merge(ws, g, &P);
    cudaStream_t s = (cudaStream_t)stream;
    MergeConsts c = consts_of(params);
    c.noise_table = reinterpret_cast<const float4 *>(noise_table_dev);
    CheckScope chk;
    chk.add(burst_dev, burst_bytes(desc));
    chk.add(motion_dev, motion_bytes(g));
    chk.add(rgb_dev, rgb_bytes(desc, scale_num, scale_den));
    chk.add(den_dev, rgb_bytes(desc, scale_num, scale_den));
    chk.add(noise_table_dev, sizeof(float4) * kNoiseLevels);
    chk.add_ws(ws, need);
    cudaError_t e = launch_merge_prep(burst_dev, motion_dev, g, c, P, s);
    if (e != cudaSuccess) return HMFSR_ERR_CUDA;
    return cuda_status(launch_merge_accum(burst_dev, motion_dev, g, P, scale_num, scale_den, rgb_dev, den_dev, s));
}

hmfsr_status hmfsr_merge_ex(const uint16_t *burst_dev, const hmfsr_burst_desc *desc, const float *motion_dev,
                            const hmfsr_merge_params *params, const hmfsr_merge_options *opts, int scale_num,
                            int scale_den, float *rgb_dev, float *den_dev, void *ws, size_t ws_bytes, void *stream) {
    hmfsr_status why;
    if (!valid_desc(desc, &why)) return why;
    if (!opts || (reinterpret_cast<uintptr_t>(opts->noise_table) & 15) || !isfinite(opts->hf_loss) || opts->hf_loss < 0.f)
        return HMFSR_ERR_INVALID_ARG;
    if (!burst_dev || !motion_dev || !rgb_dev || !aligned4(burst_dev) || !aligned8(motion_dev) || !valid_merge_params(params) ||
        !valid_scale(scale_num, scale_den))
        return HMFSR_ERR_INVALID_ARG;
    Geom g = make_geom(desc, params->tile);
    MergePlanes P;
    size_t need = carve_merge(nullptr, g, &P);
    hmfsr_status st = check_ws(ws, ws_bytes, need);
    if (st != HMFSR_OK) return st;
    carve_merge(ws, g, &P);
    cudaStream_t s = (cudaStream_t)stream;
    MergeConsts c = consts_of(params);
    c.noise_table = reinterpret_cast<const float4 *>(opts->noise_table);
    c.hf_loss = opts->hf_loss;
    CheckScope chk;
    chk.add(burst_dev, burst_bytes(desc));
    chk.add(motion_dev, motion_bytes(g));
    chk.add(rgb_dev, rgb_bytes(desc, scale_num, scale_den));
    chk.add(den_dev, rgb_bytes(desc, scale_num, scale_den));
    chk.add(opts->noise_table, sizeof(float4) * kNoiseLevels);
    chk.add_ws(ws, need);
    cudaError_t e = launch_merge_prep(burst_dev, motion_dev, g, c, P, s);
    if (e != cudaSuccess) return HMFSR_ERR_CUDA;
    return cuda_status(launch_merge_accum(burst_dev, motion_dev, g, P, scale_num, scale_den, rgb_dev, den_dev, s));
}

hmfsr_status hmfsr_merge_prepare(const uint16_t *burst_dev, const hmfsr_burst_desc *desc, const float *motion_dev,
                                 const hmfsr_merge_params *params, void *ws, size_t ws_bytes, void *stream) {
    hmfsr_status why;
    if (!valid_desc(desc, &why)) return why;
    if (!burst_dev || !motion_dev || !aligned4(burst_dev) || !aligned8(motion_dev) || !valid_merge_params(params)) return HMFSR_ERR_INVALID_ARG;
    Geom g = make_geom(desc, params->tile);
    MergePlanes P;
    const size_t need = carve_merge(nullptr, g, &P);
    hmfsr_status st = check_ws(ws, ws_bytes, need);
    if (st != HMFSR_OK) return st;
    carve_merge(ws, g, &P);
    CheckScope chk;
    chk.add(burst_dev, burst_bytes(desc));
    chk.add(motion_dev, motion_bytes(g));
    chk.add_ws(ws, need);
    return cuda_status(launch_merge_prep(burst_dev, motion_dev, g, consts_of(params), P, (cudaStream_t)stream));
}

hmfsr_status hmfsr_merge_accumulate(const uint16_t *burst_dev, const hmfsr_burst_desc *desc, const float *motion_dev,
                                    const hmfsr_merge_params *params, int scale_num, int scale_den, float *rgb_dev,
                                    float *den_dev, void *ws, size_t ws_bytes, void *stream) {
    hmfsr_status why;
    if (!valid_desc(desc, &why)) return why;
    if (!burst_dev || !motion_dev || !rgb_dev || !aligned4(burst_dev) || !aligned8(motion_dev) || !valid_merge_params(params) ||
        !valid_scale(scale_num, scale_den))
        return HMFSR_ERR_INVALID_ARG;
    Geom g = make_geom(desc, params->tile);
    MergePlanes P;
    const size_t need = carve_merge(nullptr, g, &P);
    hmfsr_status st = check_ws(ws, ws_bytes, need);
    if (st != HMFSR_OK) return st;
    carve_merge(ws, g, &P);
    CheckScope chk;
    chk.add(burst_dev, burst_bytes(desc));
    chk.add(motion_dev, motion_bytes(g));
    chk.add(rgb_dev, rgb_bytes(desc, scale_num, scale_den));
    chk.add(den_dev, rgb_bytes(desc, scale_num, scale_den));
    chk.add_ws(ws, need);
    return cuda_status(
        launch_merge_accum(burst_dev, motion_dev, g, P, scale_num, scale_den, rgb_dev, den_dev, (cudaStream_t)stream));
}

hmfsr_status hmfsr_merge_stages(const uint16_t *burst_dev, const hmfsr_burst_desc *desc, const float *motion_dev,
                                const hmfsr_merge_params *params, float *omega_dev, float *rhat_dev, void *ws,
                                size_t ws_bytes, void *stream) {
    hmfsr_status why;
    if (!valid_desc(desc, &why)) return why;
    if (!burst_dev || !motion_dev || !aligned4(burst_dev) || !aligned8(motion_dev) || !valid_merge_params(params)) return HMFSR_ERR_INVALID_ARG;
    Geom g = make_geom(desc, params->tile);
    MergePlanes P;
    size_t need = carve_merge(nullptr, g, &P);
    hmfsr_status st = check_ws(ws, ws_bytes, need);
    if (st != HMFSR_OK) return st;
    carve_merge(ws, g, &P);
    cudaStream_t s = (cudaStream_t)stream;
    const size_t hw = (size_t)g.hh * g.wh;
    CheckScope chk;
    chk.add(burst_dev, burst_bytes(desc));
    chk.add(motion_dev, motion_bytes(g));
    chk.add(omega_dev, (size_t)g.n * 3 * hw * sizeof(float));
    chk.add(rhat_dev, (size_t)g.n * hw * sizeof(float));
    chk.add_ws(ws, need);
    cudaError_t e = launch_merge_prep(burst_dev, motion_dev, g, consts_of(params), P, s);
    if (e != cudaSuccess) return HMFSR_ERR_CUDA;
    return cuda_status(launch_export_stages(g, P, omega_dev, rhat_dev, s));
}

namespace {
// the adjoint; prepared: the workspace already holds this call's merge planes (an
// hmfsr_merge with the same arguments on the same workspace), so the preparation is skipped
hmfsr_status merge_backward_impl(const uint16_t *burst_dev, const hmfsr_burst_desc *desc, const float *motion_dev,
                                 const hmfsr_merge_params *params, int scale_num, int scale_den, const float *rgb_dev,
                                 const float *den_dev, const float *grad_rgb_dev, float *grad_params_dev,
                                 float *grad_motion_dev, void *ws, size_t ws_bytes, void *stream, bool prepared) {
    hmfsr_status why;
    if (!valid_desc(desc, &why)) return why;
    if (!burst_dev || !motion_dev || !rgb_dev || !den_dev || !grad_rgb_dev || !grad_params_dev || !grad_motion_dev ||
        !aligned4(burst_dev) || !aligned8(motion_dev) || !valid_merge_params(params) || !valid_scale(scale_num, scale_den))
        return HMFSR_ERR_INVALID_ARG;
    Geom g = make_geom(desc, params->tile);
    MergePlanes P;
    BwdPlanes B;
    const int ho = (int)(((long long)desc->height * scale_num) / scale_den);
    const int wo = (int)(((long long)desc->width * scale_num) / scale_den);
    const size_t fwd = carve_merge(nullptr, g, &P);
    hmfsr_status st = check_ws(ws, ws_bytes, carve_backward(nullptr, g, ho, wo, fwd, &B));
    if (st != HMFSR_OK) return st;
    carve_merge(ws, g, &P);
    carve_backward(ws, g, ho, wo, fwd, &B);
    cudaStream_t s = (cudaStream_t)stream;
    const MergeConsts c = consts_of(params);
    SideStream *side = side_stream();
    if (!side) return HMFSR_ERR_CUDA;
    StageRange range("hmfsr merge adjoint");
    // the kernel-shape derivatives (burst only) beside the preparation; the robustness
    // derivatives (after the preparation) beside the main adjoint kernel; both joined
    // before the parts that read them
    cudaError_t e[10];
    e[0] = cudaEventRecord(side->fork, s);
    e[1] = cudaStreamWaitEvent(side->s, side->fork, 0);
    e[2] = launch_bwd_shape(burst_dev, g, B, side->s);
    e[3] = cudaEventRecord(side->join, side->s);
    e[4] = prepared ? cudaSuccess : launch_merge_prep(burst_dev, motion_dev, g, c, P, s);
    e[5] = cudaEventRecord(side->aux, s);
    e[6] = cudaStreamWaitEvent(side->s, side->aux, 0);
    e[7] = launch_bwd_robust(motion_dev, g, c, P, B, side->s);
    // the robustness part's completion, recorded after every wait above has been enqueued
    e[8] = cudaEventRecord(side->fork, side->s);
    e[9] = cudaStreamWaitEvent(s, side->join, 0);
    for (cudaError_t x : e)
        if (x != cudaSuccess) return HMFSR_ERR_CUDA;
    if (launch_bwd_main(burst_dev, motion_dev, g, c, P, B, scale_num, scale_den, rgb_dev, den_dev, grad_rgb_dev, s) !=
            cudaSuccess ||
        cudaStreamWaitEvent(s, side->fork, 0) != cudaSuccess)
        return HMFSR_ERR_CUDA;
    return cuda_status(launch_bwd_finish(g, B, scale_num, scale_den, grad_params_dev, grad_motion_dev, s));
}
}  // namespace

hmfsr_status hmfsr_merge_backward(const uint16_t *burst_dev, const hmfsr_burst_desc *desc, const float *motion_dev,
                                  const hmfsr_merge_params *params, int scale_num, int scale_den,
                                  const float *rgb_dev, const float *den_dev, const float *grad_rgb_dev,
                                  float *grad_params_dev, float *grad_motion_dev, void *ws, size_t ws_bytes,
                                  void *stream) {
    return merge_backward_impl(burst_dev, desc, motion_dev, params, scale_num, scale_den, rgb_dev, den_dev,
                               grad_rgb_dev, grad_params_dev, grad_motion_dev, ws, ws_bytes, stream, false);
}

hmfsr_status hmfsr_merge_backward_prepared(const uint16_t *burst_dev, const hmfsr_burst_desc *desc,
                                           const float *motion_dev, const hmfsr_merge_params *params, int scale_num,
                                           int scale_den, const float *rgb_dev, const float *den_dev,
                                           const float *grad_rgb_dev, float *grad_params_dev, float *grad_motion_dev,
                                           void *ws, size_t ws_bytes, void *stream) {
    return merge_backward_impl(burst_dev, desc, motion_dev, params, scale_num, scale_den, rgb_dev, den_dev,
                               grad_rgb_dev, grad_params_dev, grad_motion_dev, ws, ws_bytes, stream, true);
}


const char *hmfsr_status_string(hmfsr_status s) {
    switch (s) {
        case HMFSR_OK: return "ok";
        case HMFSR_ERR_INVALID_ARG: return "invalid argument";
        case HMFSR_ERR_UNSUPPORTED: return "unsupported";
        case HMFSR_ERR_WORKSPACE: return "workspace missing, misaligned or too small";
        case HMFSR_ERR_CUDA: return "CUDA error";
        case HMFSR_ERR_TIMEOUT: return "device wait timed out";
    }
    return "unknown status";
}

hmfsr_status hmfsr_check_status(int reset, int *line) {
#ifdef HMFSR_CHECKED
    if (!line) return HMFSR_ERR_INVALID_ARG;
    int v = 0;
    if (cudaMemcpyFromSymbol(&v, g_check_err, sizeof(int)) != cudaSuccess) return HMFSR_ERR_CUDA;
    *line = v;
    if (reset) {
        const int z = 0;
        if (cudaMemcpyToSymbol(g_check_err, &z, sizeof(int)) != cudaSuccess) return HMFSR_ERR_CUDA;
    }
    return HMFSR_OK;
#else
    (void)reset;
    (void)line;
    return HMFSR_ERR_UNSUPPORTED;
#endif
}

hmfsr_status hmfsr_check_shrink(size_t bytes) {
#ifdef HMFSR_CHECKED
    g_check_shrink = bytes;
    return HMFSR_OK;
#else
    (void)bytes;
    return HMFSR_ERR_UNSUPPORTED;
#endif
}

const char *hmfsr_version(void) { return "0.1.0"; }

}  // extern "C"
