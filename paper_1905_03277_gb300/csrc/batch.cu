// Ragged batches of bursts in one persistent launch.
//
// A plan lists, for every burst of the batch, the work items of every stage of the
// path (alignment pyramid, block matching per level, Lucas-Kanade, merge preparation,
// robustness, accumulation).  One persistent kernel -- one block of 128 threads per
// resident slot -- pops items from a global counter in an order where every item comes
// after the items it depends on; before running an item, a block waits until the stages
// it depends on have finished for that burst (per-burst, per-stage completion counters).
// The waits are bounded: after a fixed number of polls the block records
// HMFSR_ERR_TIMEOUT in a status word and every block leaves.  The run (counter reset and
// the kernel) is captured once in a CUDA graph and replayed.  An autotuner picks the
// shape of the accumulation's work item and the number of blocks per SM.
//
// Each stage runs the same device functions as the per-burst kernels (stages.cuh), so a
// batch produces bit-identical outputs to merging its bursts one by one.
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "accumulate.cuh"

namespace hmfsr {
namespace {

enum Stage {
    S_LUMA = 0, S_PREP, S_DOWN1, S_DOWN2, S_DOWN3, S_SSD3, S_SSD2, S_SSD1, S_SSD0, S_LK, S_STRENGTH, S_ROB, S_MERGE,
    S_PHANTOM, S_COUNT
};
constexpr int kBatchThreads = 128;
constexpr int kMaxDeps = 6;
// queue order: every stage after the stages it depends on
constexpr int kOrder[] = {S_LUMA, S_PREP, S_DOWN1, S_DOWN2, S_DOWN3, S_SSD3, S_SSD2, S_SSD1, S_SSD0,
                          S_LK, S_STRENGTH, S_ROB, S_MERGE};
constexpr int kLkTiles = kBatchThreads / 4;  // Lucas-Kanade tiles per sub-item (4 lanes per tile)

struct BatchBurst {
    const uint16_t *burst;
    float *motion;
    float *rgb;
    Geom g;
    MergeConsts c;
    int snum, sden, ho, wo;
    int radius[4], lk_iters;
    AlignLevels L;
    MergePlanes P;
};

struct Segment {
    int burst, stage, first, count;  // items [first, first + count) of the queue
};

struct Deps {
    int n;
    int d[kMaxDeps];
};

__device__ __host__ inline Deps stage_deps(int s) {
    Deps r{0, {0, 0, 0, 0, 0, 0}};
    auto add = [&](int x) { r.d[r.n++] = x; };
    switch (s) {
        case S_DOWN1: add(S_LUMA); break;
        case S_DOWN2: add(S_DOWN1); break;
        case S_DOWN3: add(S_DOWN2); break;
        case S_SSD3: add(S_DOWN1); add(S_DOWN2); add(S_DOWN3); break;
        case S_SSD2: add(S_DOWN1); add(S_DOWN2); add(S_DOWN3); add(S_SSD3); break;
        case S_SSD1: add(S_DOWN1); add(S_DOWN2); add(S_DOWN3); add(S_SSD2); add(S_SSD3); break;
        case S_SSD0: add(S_LUMA); add(S_DOWN3); add(S_SSD1); add(S_SSD2); add(S_SSD3); break;
        case S_LK: add(S_SSD0); break;
        case S_STRENGTH: add(S_LK); break;
        case S_ROB: add(S_PREP); add(S_STRENGTH); break;
        case S_MERGE: add(S_PREP); add(S_ROB); add(S_LK); add(S_STRENGTH); add(S_PHANTOM); break;
        default: break;
    }
    return r;
}

// level of a down-sampling or search stage
__device__ __host__ inline int stage_level(int s) {
    switch (s) {
        case S_DOWN1: case S_SSD1: return 1;
        case S_DOWN2: case S_SSD2: return 2;
        case S_DOWN3: case S_SSD3: return 3;
        default: return 0;
    }
}

// sub-items (128-thread units of work) per queue item, per stage: coarse enough that the
// queue and dependency bookkeeping of an item is small next to its work
__device__ __host__ inline int stage_k(int s) {
    switch (s) {
        case S_DOWN1: case S_DOWN2: case S_DOWN3: return 256;
        case S_LUMA: return 64;
        case S_PREP: return 16;
        case S_ROB: return 2;
        case S_LK: return 16;
        case S_MERGE: return 32;
        case S_STRENGTH: return 8;
        default: return 4;  // block matching: 128 tiles per sub-item
    }
}

// number of 128-thread sub-items of stage s of one burst (mw x mh: accumulation item shape)
__device__ __host__ inline int stage_subitems(const BatchBurst &b, int s, int mw, int mh) {
    const Geom &g = b.g;
    const int nl = b.L.n_levels;
    switch (s) {
        case S_LUMA: return div_up(g.wh, 4 * kBatchThreads) * g.hh * g.n;
        case S_PREP: return div_up(g.wh, kBatchThreads) * div_up(g.hh, stage::kPrepStrip) * g.n;
        case S_DOWN1: case S_DOWN2: case S_DOWN3: {
            const int l = stage_level(s);
            return l < nl ? div_up(b.L.lw[l], kBatchThreads) * b.L.lh[l] * g.n : 0;
        }
        case S_SSD3: case S_SSD2: case S_SSD1: case S_SSD0: {
            const int l = stage_level(s);
            return l < nl ? div_up(b.L.lty[l] * b.L.ltx[l], kBatchThreads) * g.n : 0;
        }
        case S_LK: return div_up(b.L.lty[0] * b.L.ltx[0], kLkTiles) * g.n;
        case S_STRENGTH: return div_up(g.n * g.ty * g.tx, kBatchThreads);
        case S_ROB: return div_up(g.wh, 4 * stage::kRobOut) * div_up(g.hh, stage::kRobStrip) * (g.n - 1);
        case S_MERGE:  // scale 1: blocks of 32 x 16 pixels in 2 x 2 quads (merge_quad1)
            return b.snum == b.sden ? div_up(b.wo, stage::kQuadW) * div_up(b.ho, 8 * stage::kQuadNY)
                                    : div_up(b.wo, mw) * div_up(b.ho, mh);
        default: return 0;
    }
}

__host__ inline int stage_items(const BatchBurst &b, int s, int mw, int mh) {
    return div_up(stage_subitems(b, s, mw, mh), stage_k(s));
}

template <int RAD>
__device__ __forceinline__ void run_ssd(const BatchBurst &b, int l, int tile, int f) {
    const AlignLevels &L = b.L;
    const bool top = (l == L.n_levels - 1);
    const int fsh = top ? 0 : (l == 0 ? 1 : 2);  // log2 of the factors 2, 4, 4 below level l+1
    if constexpr (RAD <= 2)
        stage::ssd_rows<8, RAD>(L.img[l], L.lh[l], L.lw[l], L.lty[l], L.ltx[l], top ? nullptr : L.vec[l + 1],
                                top ? 0 : L.lty[l + 1], top ? 0 : L.ltx[l + 1], fsh, b.g.ref, L.vec[l], tile, f);
    else
        stage::ssd<8, RAD>(L.img[l], L.lh[l], L.lw[l], L.lty[l], L.ltx[l], top ? nullptr : L.vec[l + 1],
                           top ? 0 : L.lty[l + 1], top ? 0 : L.ltx[l + 1], fsh, b.g.ref, L.vec[l], tile, f);
}

template <int SN, int SD>
__device__ __forceinline__ void run_merge(const BatchBurst &b, int X, int Y) {
    stage::merge_px<false, SN, SD>(b.burst, b.P.geo, b.g, b.P.kern, b.P.rhat,
                                   b.snum, b.sden, b.ho, b.wo, b.rgb, nullptr, X, Y);
}

// one sub-item of one stage of burst b, by all 128 threads of the block
__device__ __forceinline__ void run_sub(const BatchBurst &b, int s, int k, int tid, int mw, int mh) {
    const Geom &g = b.g;
    const float2 *mv = reinterpret_cast<const float2 *>(b.motion);
    switch (s) {
        case S_LUMA: {
            const int nx = div_up(g.wh, 4 * kBatchThreads);
            const int f = k / (nx * g.hh), r = k - f * nx * g.hh, v = r / nx, u4 = (r - v * nx) * kBatchThreads + tid;
            stage::luma0(b.burst, g.h, g.pitch, g.hh, g.wh, b.L.img[0], u4, v, f);
            break;
        }
        case S_PREP: {
            const int nx = div_up(g.wh, kBatchThreads), ny = div_up(g.hh, stage::kPrepStrip);
            const int f = k / (nx * ny), r = k - f * nx * ny, by = r / nx, bx = r - by * nx;
            stage::prep_strip(b.burst, g, b.c, b.P.s1, b.P.base_stats, b.P.kern, bx * kBatchThreads + (tid & ~31),
                              by * stage::kPrepStrip, f, tid & 31);
            break;
        }
        case S_DOWN1: case S_DOWN2: case S_DOWN3: {
            const int l = stage_level(s);
            const int nx = div_up(b.L.lw[l], kBatchThreads);
            const int f = k / (nx * b.L.lh[l]), r = k - f * nx * b.L.lh[l], y = r / nx;
            const int x = (r - y * nx) * kBatchThreads + tid;
            const int fct = (l == 1) ? 2 : 4;
            stage::down(b.L.img[l - 1], b.L.lh[l - 1], b.L.lw[l - 1], b.L.img[l], b.L.lh[l], b.L.lw[l], fct, x, y, f);
            break;
        }
        case S_SSD3: case S_SSD2: case S_SSD1: case S_SSD0: {
            const int l = stage_level(s);
            const int per = div_up(b.L.lty[l] * b.L.ltx[l], kBatchThreads);
            const int f = k / per, tile = (k - f * per) * kBatchThreads + tid;
            switch (b.radius[l]) {
                case 1: run_ssd<1>(b, l, tile, f); break;
                case 2: run_ssd<2>(b, l, tile, f); break;
                case 3: run_ssd<3>(b, l, tile, f); break;
                default: run_ssd<4>(b, l, tile, f); break;
            }
            break;
        }
        case S_LK: {
            const int per = div_up(b.L.lty[0] * b.L.ltx[0], kLkTiles);
            const int f = k / per, tile = (k - f * per) * kLkTiles + tid / 4;
            stage::lk_group<8>(b.L.img[0], b.L.lh[0], b.L.lw[0], b.L.lty[0], b.L.ltx[0], b.L.vec[0], g.ref,
                               b.lk_iters, b.motion, nullptr, tile, tid & 31, f);
            break;
        }
        case S_STRENGTH:
            stage::strength(mv, g.n, g.ty, g.tx, b.c.m_th, b.c.s1, b.c.s2, b.P.s_tile, k * kBatchThreads + tid);
            stage::geo_entry(mv, g.n, g.ty * g.tx, g.ref, 2 * b.snum, b.P.geo, k * kBatchThreads + tid);
            break;
        case S_ROB: {
            const int nx = div_up(g.wh, 4 * stage::kRobOut), ny = div_up(g.hh, stage::kRobStrip);
            const int fi = k / (nx * ny), r = k - fi * nx * ny, by = r / nx, bx = r - by * nx;
            const int f = fi < g.ref ? fi : fi + 1;  // every frame but the base frame
            stage::rob_strip(b.P.s1, b.P.base_stats, mv, b.P.s_tile, g, b.c.t, b.P.rhat,
                             (bx * 4 + (tid >> 5)) * stage::kRobOut, by * stage::kRobStrip, f, tid & 31);
            break;
        }
        case S_MERGE: {
            if (b.snum == b.sden) {
                // the per-burst kernel's layout: 4 warps of 8 x 4 threads of 2 x kQuadNY pixels
                constexpr int NY = stage::kQuadNY;
                const int nx = div_up(b.wo, stage::kQuadW), by = k / nx, bx = k - by * nx;
                const int w = tid >> 5, lane = tid & 31;
                const int qx = (w & 1) * 8 + (lane & 7), qy = (w >> 1) * 4 + (lane >> 3);
                stage::merge_quad1<false, NY>(b.burst, b.P.geo, b.g, b.P.kern, b.P.rhat, b.rgb, nullptr,
                                              bx * stage::kQuadW + 2 * qx, by * 8 * NY + NY * qy);
                break;
            }
            const int nx = div_up(b.wo, mw);
            const int by = k / nx, bx = k - by * nx;
            const int X = bx * mw + tid % mw, Y = by * mh + tid / mw;
            if (b.snum == 1 && b.sden == 1) run_merge<1, 1>(b, X, Y);
            else if (b.snum == 3 && b.sden == 2) run_merge<3, 2>(b, X, Y);
            else if (b.snum == 2 && b.sden == 1) run_merge<2, 1>(b, X, Y);
            else run_merge<0, 0>(b, X, Y);
            break;
        }
        default: break;
    }
}

// one queue item: stage_k(s) consecutive sub-items
__device__ __forceinline__ void run_item(const BatchBurst &b, int s, int k, int tid, int mw, int mh) {
    const int K = stage_k(s), nsub = stage_subitems(b, s, mw, mh);
    for (int j = 0; j < K; ++j) {
        const int sub = k * K + j;
        if (sub >= nsub) break;
        run_sub(b, s, sub, tid, mw, mh);
    }
}

__device__ __forceinline__ int load_acquire(const int *p) {
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void add_release(int *p, int v) {
    asm volatile("red.release.gpu.global.add.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

constexpr int kMaxCachedBursts = 256;

// ctrl[0]: next queue position; ctrl[1]: status (0 or HMFSR_ERR_TIMEOUT).
// prof (nullable): per stage {cycles waiting for dependencies, cycles running items,
// items}, summed over the blocks by their lead thread (SM clock cycles).
template <int MINB>
__global__ void __launch_bounds__(kBatchThreads, MINB)
    k_batch(const BatchBurst *__restrict__ bursts, const Segment *__restrict__ segs, int nseg, int total,
            int *ctrl, int *done, const int *__restrict__ totals, int mw, int mh, int spin_limit,
            unsigned long long *prof) {
    __shared__ int s_item, s_next, s_ok, s_seg;
    __shared__ long long s_t1;
    __shared__ unsigned int s_ready[kMaxCachedBursts];  // per burst: bit s set once stage s is complete
    const int tid = threadIdx.x;
    for (int i = tid; i < kMaxCachedBursts; i += kBatchThreads) s_ready[i] = 0u;
    if (tid == 0) {
        s_next = atomicAdd(&ctrl[0], 1);
        s_seg = 0;
    }
    for (;;) {
        if (tid == 0) {
            const long long t0 = prof ? clock64() : 0;
            // take the prefetched position and fetch the following one while this item runs
            const int st = *(volatile int *)&ctrl[1];
            const int item = (st != 0) ? total : s_next;
            s_item = item;
            s_next = (item < total) ? atomicAdd(&ctrl[0], 1) : total;
            int ok = 1;
            if (item < total) {
                // positions only grow, so the segment is found by scanning forward
                int sgi = s_seg;
                while (segs[sgi].first + segs[sgi].count <= item) ++sgi;
                s_seg = sgi;
                const int b = segs[sgi].burst, sidx = segs[sgi].stage;
                const Deps dp = stage_deps(sidx);
                unsigned int ready = b < kMaxCachedBursts ? s_ready[b] : 0u;
                for (int i = 0; i < dp.n && ok; ++i) {
                    const int d = dp.d[i];
                    if (ready & (1u << d)) continue;
                    const int need = totals[b * S_COUNT + d];
                    const int *cnt = &done[b * S_COUNT + d];
                    int polls = 0;
                    while (load_acquire(cnt) < need) {
                        if (++polls > spin_limit || *(volatile int *)&ctrl[1] != 0) {
                            atomicExch(&ctrl[1], (int)HMFSR_ERR_TIMEOUT);
                            ok = 0;
                            break;
                        }
                        __nanosleep(256);
                    }
                    if (ok) ready |= 1u << d;
                }
                if (b < kMaxCachedBursts) s_ready[b] = ready;
                if (prof) {
                    s_t1 = clock64();
                    atomicAdd(prof + 3 * sidx, (unsigned long long)(s_t1 - t0));
                }
            }
            s_ok = ok;
        }
        __syncthreads();
        const int item = s_item;
        if (item >= total || !s_ok) break;
        const Segment sg = segs[s_seg];
        const int b = sg.burst, s = sg.stage, k = item - sg.first;
        run_item(bursts[b], s, k, tid, mw, mh);
        __syncthreads();
        if (tid == 0) {
            add_release(&done[b * S_COUNT + s], 1);
            if (prof) {
                atomicAdd(prof + 3 * s + 1, (unsigned long long)(clock64() - s_t1));
                atomicAdd(prof + 3 * s + 2, 1ull);
            }
        }
    }
}

}  // namespace
}  // namespace hmfsr

using namespace hmfsr;

struct hmfsr_batch_plan_t {
    int nb = 0;
    std::vector<hmfsr_burst_desc> desc;
    std::vector<hmfsr_merge_params> mp;
    std::vector<hmfsr_align_params> ap;
    std::vector<int> snum, sden;
    std::vector<BatchBurst> host;  // geometry filled at creation, pointers at run time
    std::vector<size_t> burst_off; // each burst's scratch offset in the workspace
    std::vector<Segment> segs;
    std::vector<int> totals;
    int total = 0;
    size_t table_off = 0, seg_off = 0, tot_off = 0, done_off = 0, ctrl_off = 0, prof_off = 0, ws_bytes = 0;
    int profile = 0;  // the persistent kernel sums per-stage cycles (hmfsr_batch_set_profile)
    int mw = 32, mh = 4, ctas_per_sm = 0;  // accumulation item shape, blocks per SM (0: all that fit)
    int regs_variant = 1;                  // kernel build: 0 = 128, 1 = 80, 2 = 64 registers per thread
    int mode = 0;                          // 0: one persistent kernel; k > 0: graph of per-burst kernels on k streams
    int order = 0;                         // queue: 0 = stage-major, 1 = burst-major
    int spin_limit = 1 << 22;
    int inject_stall = 0;
    // device tables of the persistent mode: uploaded from pinned staging when the burst
    // pointers, the workspace or the queue change, never on a replay with the same ones
    void *staging = nullptr;       // pinned host copy of table + queue + totals
    size_t staging_bytes = 0;
    cudaEvent_t staged = nullptr;  // the last upload from staging has been copied
    bool tables_valid = false;     // the device tables match the current pointers and queue
    const void *tables_ws = nullptr;
    // captured run
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    void *graph_ws = nullptr;
    cudaStream_t graph_stream = nullptr;
    int graph_grid = 0;
};

namespace {

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// fill the item counts and the queue for the current accumulation item shape
void build_queue(hmfsr_batch_plan_t *p) {
    p->segs.clear();
    p->totals.assign((size_t)p->nb * S_COUNT, 0);
    for (int b = 0; b < p->nb; ++b) {
        for (int s = 0; s < S_COUNT; ++s) p->totals[(size_t)b * S_COUNT + s] = stage_items(p->host[b], s, p->mw, p->mh);
        p->totals[(size_t)b * S_COUNT + S_PHANTOM] = p->inject_stall ? 1 : 0;  // an item nobody runs (testing)
    }
    // stage-major: all bursts' items of one stage before the next stage; larger bursts first
    std::vector<int> order(p->nb);
    for (int b = 0; b < p->nb; ++b) order[b] = b;
    std::stable_sort(order.begin(), order.end(), [&](int a, int c) {
        return (long long)p->desc[a].height * p->desc[a].width * p->desc[a].n_frames >
               (long long)p->desc[c].height * p->desc[c].width * p->desc[c].n_frames;
    });
    int first = 0;
    auto push = [&](int b, int s) {
        const int cnt = p->totals[(size_t)b * S_COUNT + s];
        if (cnt == 0) return;
        p->segs.push_back(Segment{b, s, first, cnt});
        first += cnt;
    };
    // any order that keeps each burst's stages in kOrder is topological: a burst's stages
    // only wait on its own earlier stages
    const int nst = (int)(sizeof(kOrder) / sizeof(kOrder[0]));
    if (p->order == 0) {
        for (int si = 0; si < nst; ++si)
            for (int b : order) push(b, kOrder[si]);
    } else if (p->order == 1) {
        for (int b : order)
            for (int si = 0; si < nst; ++si) push(b, kOrder[si]);
    } else {
        // wavefront: the r-th burst's stage si is queued at step si + 2 r, so a burst's
        // stages stay close in time (its planes still in L2) while other bursts' work
        // fills its stage boundaries
        for (int step = 0; step < nst + 2 * p->nb; ++step)
            for (int r = 0; r < p->nb; ++r) {
                const int si = step - 2 * r;
                if (si >= 0 && si < nst) push(order[r], kOrder[si]);
            }
    }
    p->total = first;
}

void drop_graph(hmfsr_batch_plan_t *p) {
    p->tables_valid = false;
    if (p->exec) cudaGraphExecDestroy(p->exec);
    if (p->graph) cudaGraphDestroy(p->graph);
    p->exec = nullptr;
    p->graph = nullptr;
}

bool batch_desc_ok(const hmfsr_burst_desc &d, const hmfsr_merge_params &m, const hmfsr_align_params &a, int sn, int sd) {
    if (d.n_frames < 1 || d.height < 32 || d.width < 32 || (d.height & 1) || (d.width & 1) || d.pitch_elems < d.width ||
        (d.pitch_elems & 1) || d.ref < 0 || d.ref >= d.n_frames || d.cfa != 0 || d.black_level != 0 ||
        d.white_level < 1 || d.white_level > 7281 || d.height > 65536 || d.width > 65536 ||
        (long long)d.height * d.pitch_elems >= (1LL << 31))
        return false;
    if (m.tile != 16 || a.tile != 16 || a.n_levels < 1 || a.n_levels > 4 || a.lk_iters < 0 || a.lk_iters > 16)
        return false;
    for (int l = 0; l < 4; ++l)
        if (a.radius[l] < 1 || a.radius[l] > 4) return false;
    if (!(m.k_detail > 0.f && m.k_denoise > 0.f && m.d_tr > 0.f && m.k_stretch > 0.f && m.k_shrink > 0.f &&
          m.noise_a >= 0.f && m.noise_b >= 0.f))
        return false;
    return sn >= 1 && sd >= 1 && sn <= 8 && sd <= 8 && sn >= sd && sn <= 4 * sd;
}

}  // namespace

extern "C" {

hmfsr_status hmfsr_batch_plan_create(const hmfsr_burst_desc *descs, int n_bursts, const hmfsr_merge_params *mparams,
                                     const hmfsr_align_params *aparams, const int *scale_num, const int *scale_den,
                                     hmfsr_batch_plan *out) {
    if (!out) return HMFSR_ERR_INVALID_ARG;
    *out = nullptr;
    if (!descs || !mparams || !aparams || !scale_num || !scale_den || n_bursts < 1 || n_bursts > 4096)
        return HMFSR_ERR_INVALID_ARG;
    for (int b = 0; b < n_bursts; ++b)
        if (!batch_desc_ok(descs[b], mparams[b], aparams[b], scale_num[b], scale_den[b])) return HMFSR_ERR_INVALID_ARG;
    hmfsr_batch_plan_t *p = new hmfsr_batch_plan_t();
    p->nb = n_bursts;
    p->desc.assign(descs, descs + n_bursts);
    p->mp.assign(mparams, mparams + n_bursts);
    p->ap.assign(aparams, aparams + n_bursts);
    p->snum.assign(scale_num, scale_num + n_bursts);
    p->sden.assign(scale_den, scale_den + n_bursts);
    p->host.resize(n_bursts);
    p->burst_off.resize(n_bursts);
    size_t off = 0;
    // control block first: table, queue, totals, counters
    const size_t table_bytes = sizeof(BatchBurst) * n_bursts;
    const size_t seg_bytes = sizeof(Segment) * (size_t)n_bursts * S_COUNT;
    const size_t tot_bytes = sizeof(int) * (size_t)n_bursts * S_COUNT;
    p->table_off = off; off = align256(off + table_bytes);
    p->seg_off = off; off = align256(off + seg_bytes);
    p->tot_off = off; off = align256(off + tot_bytes);
    p->done_off = off; off = align256(off + tot_bytes);
    p->ctrl_off = off; off = align256(off + 2 * sizeof(int));
    p->prof_off = off; off = align256(off + 3 * S_COUNT * sizeof(unsigned long long));
    for (int b = 0; b < n_bursts; ++b) {
        BatchBurst &bb = p->host[b];
        memset(&bb, 0, sizeof(bb));
        const hmfsr_burst_desc &d = descs[b];
        Geom &g = bb.g;
        g.n = d.n_frames; g.h = d.height; g.w = d.width; g.pitch = d.pitch_elems; g.ref = d.ref; g.wl = d.white_level;
        g.hh = d.height / 2; g.wh = d.width / 2; g.tile = 16; g.ty = div_up(d.height, 16); g.tx = div_up(d.width, 16);
        const hmfsr_merge_params &m = mparams[b];
        bb.c.k_detail = m.k_detail; bb.c.k_denoise = m.k_denoise; bb.c.d_th = m.d_th; bb.c.d_tr = m.d_tr;
        bb.c.k_stretch = m.k_stretch; bb.c.k_shrink = m.k_shrink; bb.c.t = m.t; bb.c.s1 = m.s1; bb.c.s2 = m.s2;
        bb.c.m_th = m.m_th; bb.c.noise_a = m.noise_a; bb.c.noise_b = m.noise_b;
        bb.snum = scale_num[b]; bb.sden = scale_den[b];
        bb.ho = (int)(((long long)d.height * bb.snum) / bb.sden);
        bb.wo = (int)(((long long)d.width * bb.snum) / bb.sden);
        for (int l = 0; l < 4; ++l) bb.radius[l] = aparams[b].radius[l];
        bb.lk_iters = aparams[b].lk_iters;
        // alignment levels (same rule as hmfsr_align)
        static const int fac[3] = {2, 4, 4};
        AlignLevels &L = bb.L;
        L.lh[0] = g.hh; L.lw[0] = g.wh;
        int nl = 1;
        while (nl < aparams[b].n_levels && nl < 4) {
            const int nh = L.lh[nl - 1] / fac[nl - 1], nw = L.lw[nl - 1] / fac[nl - 1];
            if (nh < 16 || nw < 16) break;
            L.lh[nl] = nh; L.lw[nl] = nw;
            ++nl;
        }
        L.n_levels = nl;
        p->burst_off[b] = off;
        for (int l = 0; l < nl; ++l) {
            L.lty[l] = div_up(L.lh[l], 8);
            L.ltx[l] = div_up(L.lw[l], 8);
            off = align256(off + sizeof(uint16_t) * (size_t)g.n * L.lh[l] * L.lw[l]);
            off = align256(off + sizeof(int2) * (size_t)g.n * L.lty[l] * L.ltx[l]);
        }
        const size_t hw = (size_t)g.hh * g.wh;
        off = align256(off + sizeof(uint2) * g.n * hw);
        off = align256(off + sizeof(float4) * hw);
        off = align256(off + sizeof(float4) * g.n * hw);
        off = align256(off + sizeof(float) * g.n * hw);
        off = align256(off + sizeof(float) * (size_t)g.n * g.ty * g.tx);
        off = align256(off + sizeof(int4) * (size_t)g.n * g.ty * g.tx);
        off = align256(off + sizeof(float) * (size_t)g.n * g.ty * g.tx * 2);  // motion when the caller gives none
    }
    p->ws_bytes = off;
    build_queue(p);
    *out = p;
    return HMFSR_OK;
}

size_t hmfsr_batch_workspace_size(hmfsr_batch_plan plan) { return plan ? plan->ws_bytes : 0; }

hmfsr_status hmfsr_batch_set_mode(hmfsr_batch_plan plan, int streams);

hmfsr_status hmfsr_batch_configure(hmfsr_batch_plan plan, int merge_tile_w, int ctas_per_sm, int regs_variant,
                                   int queue_order, int spin_limit, int inject_stall) {
    if (!plan || merge_tile_w < 1 || merge_tile_w > kBatchThreads || kBatchThreads % merge_tile_w != 0 ||
        ctas_per_sm < 0 || ctas_per_sm > 16 || spin_limit < 1 || regs_variant < 0 || regs_variant > 2 ||
        queue_order < 0 || queue_order > 2)
        return HMFSR_ERR_INVALID_ARG;
    plan->regs_variant = regs_variant;
    plan->order = queue_order;
    plan->mw = merge_tile_w;
    plan->mh = kBatchThreads / merge_tile_w;
    plan->ctas_per_sm = ctas_per_sm;
    plan->spin_limit = spin_limit;
    plan->inject_stall = inject_stall ? 1 : 0;
    build_queue(plan);
    drop_graph(plan);
    return HMFSR_OK;
}

hmfsr_status hmfsr_batch_run(hmfsr_batch_plan plan, const uint16_t *const *bursts_dev, float *const *motion_dev,
                             float *const *rgb_dev, void *ws, size_t ws_bytes, void *stream) {
    if (!plan || !bursts_dev || !rgb_dev) return HMFSR_ERR_INVALID_ARG;
    if (!ws || ws_bytes < plan->ws_bytes || (reinterpret_cast<uintptr_t>(ws) & 255)) return HMFSR_ERR_WORKSPACE;
    char *base = static_cast<char *>(ws);
    bool changed = !plan->tables_valid || plan->tables_ws != ws;
    for (int b = 0; b < plan->nb; ++b) {
        if (!bursts_dev[b] || !rgb_dev[b] || (reinterpret_cast<uintptr_t>(bursts_dev[b]) & 3)) return HMFSR_ERR_INVALID_ARG;
        BatchBurst &bb = plan->host[b];
        const float *old_motion = bb.motion;
        changed = changed || bb.burst != bursts_dev[b] || bb.rgb != rgb_dev[b];
        bb.burst = bursts_dev[b];
        bb.rgb = rgb_dev[b];
        size_t off = plan->burst_off[b];
        const Geom &g = bb.g;
        for (int l = 0; l < bb.L.n_levels; ++l) {
            bb.L.img[l] = reinterpret_cast<uint16_t *>(base + off);
            off = align256(off + sizeof(uint16_t) * (size_t)g.n * bb.L.lh[l] * bb.L.lw[l]);
            bb.L.vec[l] = reinterpret_cast<int2 *>(base + off);
            off = align256(off + sizeof(int2) * (size_t)g.n * bb.L.lty[l] * bb.L.ltx[l]);
        }
        const size_t hw = (size_t)g.hh * g.wh;
        bb.P.s1 = reinterpret_cast<uint2 *>(base + off); off = align256(off + sizeof(uint2) * g.n * hw);
        bb.P.base_stats = reinterpret_cast<float4 *>(base + off); off = align256(off + sizeof(float4) * hw);
        bb.P.kern = reinterpret_cast<float4 *>(base + off); off = align256(off + sizeof(float4) * g.n * hw);
        bb.P.rhat = reinterpret_cast<float *>(base + off); off = align256(off + sizeof(float) * g.n * hw);
        bb.P.s_tile = reinterpret_cast<float *>(base + off); off = align256(off + sizeof(float) * (size_t)g.n * g.ty * g.tx);
        bb.P.geo = reinterpret_cast<int4 *>(base + off); off = align256(off + sizeof(int4) * (size_t)g.n * g.ty * g.tx);
        float *own_motion = reinterpret_cast<float *>(base + off);
        bb.motion = (motion_dev && motion_dev[b]) ? motion_dev[b] : own_motion;
        if (reinterpret_cast<uintptr_t>(bb.motion) & 7) return HMFSR_ERR_INVALID_ARG;
        changed = changed || bb.motion != old_motion;
    }
    cudaStream_t s = (cudaStream_t)stream;
    if (plan->mode > 0) {
        // graph of each burst's own kernel sequence (the per-burst path), bursts spread
        // over plan->mode parallel branches
        if (!plan->exec || plan->graph_ws != ws || plan->graph_stream != s || plan->graph_grid != -plan->mode) {
            drop_graph(plan);
            const int ns = plan->mode;
            std::vector<cudaStream_t> br(ns);
            std::vector<cudaEvent_t> ev(ns + 1);
            cudaStream_t cap;
            cudaError_t e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
            for (int i = 0; i < ns && e == cudaSuccess; ++i) e = cudaStreamCreateWithFlags(&br[i], cudaStreamNonBlocking);
            for (int i = 0; i <= ns && e == cudaSuccess; ++i) e = cudaEventCreateWithFlags(&ev[i], cudaEventDisableTiming);
            if (e == cudaSuccess) e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
            if (e == cudaSuccess) {
                // zero the status word so hmfsr_batch_wait reports OK
                cudaMemsetAsync(base + plan->ctrl_off, 0, 2 * sizeof(int), cap);
                cudaEventRecord(ev[ns], cap);
                for (int i = 0; i < ns; ++i) cudaStreamWaitEvent(br[i], ev[ns], 0);
                std::vector<int> order(plan->nb);
                for (int b = 0; b < plan->nb; ++b) order[b] = b;
                std::stable_sort(order.begin(), order.end(), [&](int a, int c) {
                    return (long long)plan->desc[a].height * plan->desc[a].width * plan->desc[a].n_frames >
                           (long long)plan->desc[c].height * plan->desc[c].width * plan->desc[c].n_frames;
                });
                for (int r = 0; r < plan->nb; ++r) {
                    const int b = order[r];
                    const BatchBurst &bb = plan->host[b];
                    cudaStream_t bs = br[r % ns];
                    launch_align(bb.burst, bb.g, plan->ap[b], bb.L, bb.motion, nullptr, bs);
                    launch_merge_prep(bb.burst, bb.motion, bb.g, bb.c, bb.P, bs);
                    launch_merge_accum(bb.burst, bb.motion, bb.g, bb.P, bb.snum, bb.sden, bb.rgb, nullptr, bs);
                }
                for (int i = 0; i < ns; ++i) {
                    cudaEventRecord(ev[i], br[i]);
                    cudaStreamWaitEvent(cap, ev[i], 0);
                }
                e = cudaStreamEndCapture(cap, &plan->graph);
            }
            if (e == cudaSuccess) e = cudaGraphInstantiate(&plan->exec, plan->graph, 0);
            for (int i = 0; i <= ns; ++i) cudaEventDestroy(ev[i]);
            for (int i = 0; i < ns; ++i) cudaStreamDestroy(br[i]);
            cudaStreamDestroy(cap);
            if (e != cudaSuccess) {
                drop_graph(plan);
                return HMFSR_ERR_CUDA;
            }
            plan->graph_ws = ws;
            plan->graph_stream = s;
            plan->graph_grid = -plan->mode;
        }
        return cudaGraphLaunch(plan->exec, s) == cudaSuccess ? HMFSR_OK : HMFSR_ERR_CUDA;
    }
    // tables: uploaded when the pointers, the workspace or the queue changed since the
    // last upload, as one copy from pinned staging on the stream (ordered before the
    // kernel); the host waits only if the previous upload from staging is still pending
    if (changed) {
        const size_t tb = sizeof(BatchBurst) * plan->nb, sb = sizeof(Segment) * plan->segs.size();
        const size_t cb = sizeof(int) * plan->totals.size();
        const size_t need = plan->tot_off + cb;  // table, queue and totals, as laid out in ws
        if (plan->staging_bytes < need) {
            if (plan->staged && cudaEventSynchronize(plan->staged) != cudaSuccess) return HMFSR_ERR_CUDA;
            if (plan->staging) cudaFreeHost(plan->staging);
            plan->staging = nullptr;
            plan->staging_bytes = 0;
            if (cudaHostAlloc(&plan->staging, need, cudaHostAllocDefault) != cudaSuccess) return HMFSR_ERR_CUDA;
            plan->staging_bytes = need;
        }
        if (!plan->staged && cudaEventCreateWithFlags(&plan->staged, cudaEventDisableTiming) != cudaSuccess)
            return HMFSR_ERR_CUDA;
        if (cudaEventSynchronize(plan->staged) != cudaSuccess) return HMFSR_ERR_CUDA;
        char *st = static_cast<char *>(plan->staging);
        memcpy(st + plan->table_off, plan->host.data(), tb);
        memcpy(st + plan->seg_off, plan->segs.data(), sb);
        memcpy(st + plan->tot_off, plan->totals.data(), cb);
        if (cudaMemcpyAsync(base, st, need, cudaMemcpyHostToDevice, s) != cudaSuccess ||
            cudaEventRecord(plan->staged, s) != cudaSuccess)
            return HMFSR_ERR_CUDA;
        plan->tables_valid = true;
        plan->tables_ws = ws;
    }
    // persistent grid: the blocks that fit on the device (or the tuned count per SM)
    using KernelFn = void (*)(const BatchBurst *, const Segment *, int, int, int *, int *, const int *, int, int, int,
                              unsigned long long *);
    const KernelFn kernel = plan->regs_variant == 0 ? k_batch<4> : (plan->regs_variant == 1 ? k_batch<6> : k_batch<8>);
    int dev = 0, nsm = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kBatchThreads, 0) != cudaSuccess || per_sm < 1)
        return HMFSR_ERR_CUDA;
    if (plan->ctas_per_sm > 0) per_sm = std::min(per_sm, plan->ctas_per_sm);
    const int grid = std::max(1, std::min(nsm * per_sm, plan->total));
    if (!plan->exec || plan->graph_ws != ws || plan->graph_stream != s || plan->graph_grid != grid) {
        drop_graph(plan);
        cudaStream_t cap;
        if (cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) != cudaSuccess) return HMFSR_ERR_CUDA;
        cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            // completion counters, control words and the stage profile start at zero
            const size_t ctr_bytes = (size_t)(plan->prof_off - plan->done_off) + 3 * S_COUNT * sizeof(unsigned long long);
            cudaMemsetAsync(base + plan->done_off, 0, ctr_bytes, cap);
            kernel<<<grid, kBatchThreads, 0, cap>>>(
                reinterpret_cast<const BatchBurst *>(base + plan->table_off),
                reinterpret_cast<const Segment *>(base + plan->seg_off), (int)plan->segs.size(), plan->total,
                reinterpret_cast<int *>(base + plan->ctrl_off), reinterpret_cast<int *>(base + plan->done_off),
                reinterpret_cast<const int *>(base + plan->tot_off), plan->mw, plan->mh, plan->spin_limit,
                plan->profile ? reinterpret_cast<unsigned long long *>(base + plan->prof_off) : nullptr);
            e = cudaStreamEndCapture(cap, &plan->graph);
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&plan->exec, plan->graph, 0);
        cudaStreamDestroy(cap);
        if (e != cudaSuccess) {
            drop_graph(plan);
            return HMFSR_ERR_CUDA;
        }
        plan->graph_ws = ws;
        plan->graph_stream = s;
        plan->graph_grid = grid;
    }
    return cudaGraphLaunch(plan->exec, s) == cudaSuccess ? HMFSR_OK : HMFSR_ERR_CUDA;
}

hmfsr_status hmfsr_batch_set_mode(hmfsr_batch_plan plan, int streams) {
    if (!plan || streams < 0 || streams > 16) return HMFSR_ERR_INVALID_ARG;
    plan->mode = streams;
    drop_graph(plan);
    return HMFSR_OK;
}

hmfsr_status hmfsr_batch_wait(hmfsr_batch_plan plan, void *ws, void *stream) {
    if (!plan || !ws) return HMFSR_ERR_INVALID_ARG;
    int status = 0;
    cudaStream_t s = (cudaStream_t)stream;
    if (cudaMemcpyAsync(&status, static_cast<char *>(ws) + plan->ctrl_off + sizeof(int), sizeof(int),
                        cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return HMFSR_ERR_CUDA;
    return status == 0 ? HMFSR_OK : (hmfsr_status)status;
}

hmfsr_status hmfsr_batch_set_profile(hmfsr_batch_plan plan, int enable) {
    if (!plan) return HMFSR_ERR_INVALID_ARG;
    plan->profile = enable ? 1 : 0;
    drop_graph(plan);
    return HMFSR_OK;
}

hmfsr_status hmfsr_batch_stage_profile(hmfsr_batch_plan plan, const void *ws, unsigned long long *out, int n_out,
                                       void *stream) {
    if (!plan || !ws || !out || n_out < 3 * (int)S_COUNT) return HMFSR_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    if (cudaMemcpyAsync(out, static_cast<const char *>(ws) + plan->prof_off, 3 * S_COUNT * sizeof(unsigned long long),
                        cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return HMFSR_ERR_CUDA;
    return HMFSR_OK;
}

hmfsr_status hmfsr_batch_vectors(hmfsr_batch_plan plan, const void *ws, int burst, int32_t *motion_int_dev,
                                 void *stream) {
    if (!plan || !ws || !motion_int_dev || burst < 0 || burst >= plan->nb ||
        (reinterpret_cast<uintptr_t>(motion_int_dev) & 3))
        return HMFSR_ERR_INVALID_ARG;
    // level 0's vectors follow level 0's image in the burst's part of the workspace
    const BatchBurst &bb = plan->host[burst];
    const size_t off = plan->burst_off[burst] + align256(sizeof(uint16_t) * (size_t)bb.g.n * bb.L.lh[0] * bb.L.lw[0]);
    const size_t bytes = sizeof(int2) * (size_t)bb.g.n * bb.L.lty[0] * bb.L.ltx[0];
    return cudaMemcpyAsync(motion_int_dev, static_cast<const char *>(ws) + off, bytes, cudaMemcpyDeviceToDevice,
                           (cudaStream_t)stream) == cudaSuccess ? HMFSR_OK : HMFSR_ERR_CUDA;
}

hmfsr_status hmfsr_batch_tune(hmfsr_batch_plan plan, const uint16_t *const *bursts_dev, float *const *motion_dev,
                              float *const *rgb_dev, void *ws, size_t ws_bytes, void *stream, float *best_ms,
                              float *tune_log) {
    if (!plan) return HMFSR_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return HMFSR_ERR_CUDA;
    // candidates: {mode, merge tile width, register variant, queue order}
    static const int kCand[][4] = {{0, 32, 0, 0}, {0, 16, 0, 0}, {0, 32, 1, 0}, {0, 32, 2, 0},
                                   {0, 32, 0, 2}, {2, 32, 0, 0}, {4, 32, 0, 0}, {8, 32, 0, 0}};
    float best = 1e30f;
    int best_i = 0;
    hmfsr_status st = HMFSR_OK;
    for (int ci = 0; ci < (int)(sizeof(kCand) / sizeof(kCand[0])) && st == HMFSR_OK; ++ci) {
        st = hmfsr_batch_configure(plan, kCand[ci][1], 0, kCand[ci][2], kCand[ci][3], plan->spin_limit, 0);
        if (st == HMFSR_OK) st = hmfsr_batch_set_mode(plan, kCand[ci][0]);
        for (int rep = 0; rep < 2 && st == HMFSR_OK; ++rep) {
            // the first run builds the graph; the second is timed
            if (rep == 1) cudaEventRecord(e0, s);
            st = hmfsr_batch_run(plan, bursts_dev, motion_dev, rgb_dev, ws, ws_bytes, stream);
            if (rep == 1) cudaEventRecord(e1, s);
            if (st == HMFSR_OK) st = hmfsr_batch_wait(plan, ws, stream);
        }
        float ms = 0.f;
        if (st == HMFSR_OK && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess) {
            if (tune_log) tune_log[ci] = ms;
            if (ms < best) {
                best = ms;
                best_i = ci;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != HMFSR_OK) return st;
    if (best_ms) *best_ms = best;
    st = hmfsr_batch_configure(plan, kCand[best_i][1], 0, kCand[best_i][2], kCand[best_i][3], plan->spin_limit, 0);
    return st == HMFSR_OK ? hmfsr_batch_set_mode(plan, kCand[best_i][0]) : st;
}

void hmfsr_batch_free(hmfsr_batch_plan plan) {
    if (!plan) return;
    drop_graph(plan);
    if (plan->staged) {
        cudaEventSynchronize(plan->staged);
        cudaEventDestroy(plan->staged);
    }
    if (plan->staging) cudaFreeHost(plan->staging);
    delete plan;
}

}  // extern "C"
