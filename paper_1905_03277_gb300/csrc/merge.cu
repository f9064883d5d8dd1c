// Merge (Sec. 5): per-frame kernel covariances (Eq. 3-4 + supplement S.1), robustness
// (Eq. 5-9) and the kernel-regression accumulation (Eq. 1-2) with a fused
// normalisation -- the per-burst kernels.  Their bodies (and the numerical design notes)
// live in stages.cuh, shared with the batched persistent kernel.
#include <atomic>

#include "accumulate.cuh"

namespace hmfsr {
namespace {

using stage::kMergeW;
using stage::kMergeH;

// 4 warps side by side: 128 texel columns x `rows` rows of frame f0 + blockIdx.z
__global__ void __launch_bounds__(128) k_prep(const uint16_t *__restrict__ burst, Geom g, MergeConsts c,
                                              uint2 *__restrict__ s1, float4 *__restrict__ base_stats,
                                              float4 *__restrict__ kern, int rows, int f0) {
    stage::prep_strip(burst, g, c, s1, base_stats, kern, blockIdx.x * 128 + (threadIdx.x & ~31),
                      blockIdx.y * rows, f0 + blockIdx.z, threadIdx.x & 31, rows);
}

__global__ void k_strength(const float2 *__restrict__ motion, int n, int ty, int tx, float m_th, float s1, float s2,
                           float *__restrict__ s_tile) {
    stage::strength(motion, n, ty, tx, m_th, s1, s2, s_tile, blockIdx.x * blockDim.x + threadIdx.x);
}

// 4 warps side by side: 4 x kRobOut texel columns x `rows` rows of one frame
// (blockIdx.z runs over the frames other than the base frame)
// kHF: with the high-frequency rejection (hf_flag, m_th)
template <bool kHF>
__global__ void __launch_bounds__(128) k_rob(const uint2 *__restrict__ s1, const float4 *__restrict__ base_stats,
                                             const float2 *__restrict__ motion, const float *__restrict__ s_tile,
                                             Geom g, float t_thr, float *__restrict__ rhat,
                                             const unsigned char *__restrict__ hf_flag, float m_th, int rows) {
    const int frame = (int)blockIdx.z < g.ref ? (int)blockIdx.z : (int)blockIdx.z + 1;
    stage::rob_strip<kHF>(s1, base_stats, motion, s_tile, g, t_thr, rhat,
                          (blockIdx.x * 4 + (threadIdx.x >> 5)) * stage::kRobOut, blockIdx.y * rows, frame,
                          threadIdx.x & 31, hf_flag, m_th, rows);
}

__global__ void k_hf_flag(const uint16_t *__restrict__ burst, const uint2 *__restrict__ s1, Geom g, float kappa,
                          unsigned char *__restrict__ flag) {
    stage::hf_flag_px(burst, s1, g, kappa, flag, blockIdx.x * blockDim.x + threadIdx.x, blockIdx.y);
}

__global__ void k_geo(const float2 *__restrict__ motion, int n, int ntl, int ref, int Q, int4 *__restrict__ geo) {
    stage::geo_entry(motion, n, ntl, ref, Q, geo, blockIdx.x * blockDim.x + threadIdx.x);
}

template <bool kDen, int SN, int SD>
__global__ void __launch_bounds__(kMergeW *kMergeH, 8) k_merge(const uint16_t *__restrict__ burst,
                                                           const int4 *__restrict__ geo, Geom g,
                                                           const float4 *__restrict__ kern,
                                                           const float *__restrict__ rhat_planes, int snum_rt,
                                                           int sden_rt, int ho, int wo, float *__restrict__ rgb,
                                                           float *__restrict__ den_out) {
    stage::merge_px<kDen, SN, SD>(burst, geo, g, kern, rhat_planes, snum_rt, sden_rt, ho, wo, rgb, den_out,
                                  blockIdx.x * kMergeW + threadIdx.x, blockIdx.y * kMergeH + threadIdx.y);
}

// scale 1: one thread per 2 x kQuadNY output pixels; 4 warps of 8 x 4 threads (16 x
// 4 kQuadNY pixels, so that a warp lies inside one 16-pixel motion tile), the block
// 32 x 8 kQuadNY pixels
template <bool kDen, int NY>
__global__ void __launch_bounds__(128, (NY == 2 ? 4 : 5)) k_merge_q1(const uint16_t *__restrict__ burst,
                                                                    const int4 *__restrict__ geo, Geom g,
                                                                    const float4 *__restrict__ kern,
                                                                    const float *__restrict__ rhat_planes,
                                                                    float *__restrict__ rgb, float *__restrict__ den_out) {
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int qx = (w & 1) * 8 + (lane & 7), qy = (w >> 1) * 4 + (lane >> 3);
    stage::merge_quad1<kDen, NY>(burst, geo, g, kern, rhat_planes, rgb, den_out, blockIdx.x * stage::kQuadW + 2 * qx,
                                 blockIdx.y * 8 * NY + NY * qy);
}

// The same accumulation for one chunk of frames (bounded-memory merge): the running sums
// come from and go to the state buffer of `io` (stage::ChunkIO).
template <bool kDen, int SN, int SD>
__global__ void __launch_bounds__(kMergeW *kMergeH, 8) k_merge_chunk(const uint16_t *__restrict__ burst,
                                                                 const int4 *__restrict__ geo, Geom g,
                                                                 const float4 *__restrict__ kern,
                                                                 const float *__restrict__ rhat_planes, int snum_rt,
                                                                 int sden_rt, int ho, int wo, float *__restrict__ rgb,
                                                                 float *__restrict__ den_out, stage::ChunkIO io) {
    stage::merge_px<kDen, SN, SD, true>(burst, geo, g, kern, rhat_planes, snum_rt, sden_rt, ho, wo, rgb, den_out,
                                        blockIdx.x * kMergeW + threadIdx.x, blockIdx.y * kMergeH + threadIdx.y, io);
}

template <bool kDen, int NY>
__global__ void __launch_bounds__(128, (NY == 2 ? 4 : 5)) k_merge_q1_chunk(const uint16_t *__restrict__ burst,
                                                                          const int4 *__restrict__ geo, Geom g,
                                                                          const float4 *__restrict__ kern,
                                                                          const float *__restrict__ rhat_planes,
                                                                          float *__restrict__ rgb,
                                                                          float *__restrict__ den_out,
                                                                          stage::ChunkIO io) {
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int qx = (w & 1) * 8 + (lane & 7), qy = (w >> 1) * 4 + (lane >> 3);
    stage::merge_quad1<kDen, NY, true>(burst, geo, g, kern, rhat_planes, rgb, den_out,
                                       blockIdx.x * stage::kQuadW + 2 * qx, blockIdx.y * 8 * NY + NY * qy, io);
}

template <bool kDen>
static void launch_k_merge_chunk(dim3 grid, cudaStream_t s, const uint16_t *burst, const int4 *mv, const Geom &g,
                                 const MergePlanes &P, int snum, int sden, int ho, int wo, float *rgb, float *den,
                                 const stage::ChunkIO &io) {
    const dim3 block(kMergeW, kMergeH);
    if (snum == sden)
        k_merge_q1_chunk<kDen, stage::kQuadNY>
            <<<dim3(div_up(wo, stage::kQuadW), div_up(ho, 8 * stage::kQuadNY)), 128, 0, s>>>(burst, mv, g, P.kern,
                                                                                             P.rhat, rgb, den, io);
    else if (snum == 3 && sden == 2)
        k_merge_chunk<kDen, 3, 2><<<grid, block, 0, s>>>(burst, mv, g, P.kern, P.rhat, snum, sden, ho, wo, rgb, den, io);
    else if (snum == 2 && sden == 1)
        k_merge_chunk<kDen, 2, 1><<<grid, block, 0, s>>>(burst, mv, g, P.kern, P.rhat, snum, sden, ho, wo, rgb, den, io);
    else
        k_merge_chunk<kDen, 0, 0><<<grid, block, 0, s>>>(burst, mv, g, P.kern, P.rhat, snum, sden, ho, wo, rgb, den, io);
}

template <bool kDen>
static void launch_k_merge(dim3 grid, cudaStream_t s, const uint16_t *burst, const int4 *mv, const Geom &g,
                           const MergePlanes &P, int snum, int sden, int ho, int wo, float *rgb, float *den) {
    const dim3 block(kMergeW, kMergeH);
    if (snum == sden)
        k_merge_q1<kDen, stage::kQuadNY><<<dim3(div_up(wo, stage::kQuadW), div_up(ho, 8 * stage::kQuadNY)), 128, 0, s>>>(
            burst, mv, g, P.kern, P.rhat, rgb, den);
    else if (snum == 3 && sden == 2)
        k_merge<kDen, 3, 2><<<grid, block, 0, s>>>(burst, mv, g, P.kern, P.rhat, snum, sden, ho, wo, rgb, den);
    else if (snum == 2 && sden == 1)
        k_merge<kDen, 2, 1><<<grid, block, 0, s>>>(burst, mv, g, P.kern, P.rhat, snum, sden, ho, wo, rgb, den);
    else
        k_merge<kDen, 0, 0><<<grid, block, 0, s>>>(burst, mv, g, P.kern, P.rhat, snum, sden, ho, wo, rgb, den);
}

// --------------------------------------------------------------------------------------
// stage export (testing): Omega entries and Rhat planes
// --------------------------------------------------------------------------------------
__global__ void k_export(const float4 *__restrict__ kern, const float *__restrict__ rhat, int n, int ref, size_t hw,
                         float *__restrict__ omega, float *__restrict__ rhat_out) {
    size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    int f = blockIdx.y;
    if (i >= hw) return;
    if (omega) {
        const float4 t = HMFSR_LD(kern + (size_t)f * hw + i);
        float *o = omega + (size_t)f * 3 * hw;
        HMFSR_ST(o + i, t.x + t.y * t.z * t.z);
        HMFSR_ST(o + hw + i, t.y * t.z * t.w);
        HMFSR_ST(o + 2 * hw + i, t.x + t.y * t.w * t.w);
    }
    if (rhat_out) HMFSR_ST(rhat_out + (size_t)f * hw + i, (f == ref) ? 1.f : HMFSR_LD(rhat + (size_t)f * hw + i));
}

// --------------------------------------------------------------------------------------
// strip heights.  A strip kernel's blocks run in waves of (resident blocks per SM) x
// (SMs).  For the latency-bound k_rob a last wave that is only partly filled costs as
// long as a full one: of the even heights in [lo, hi], take the one with the least
// waves x (rows + halo), the rows every block walks, halo included (strip_rows).  The
// occupancy of each kernel is queried once per device; if a query fails, the default
// height stands.
// --------------------------------------------------------------------------------------
enum StripKernel { SK_PREP = 0, SK_ROB = 1, SK_ROB_HF = 2, SK_COUNT = 3 };
constexpr int kMaxDevices = 64;
std::atomic<int> g_strip_slots[SK_COUNT][kMaxDevices];  // resident blocks on the device, 0: not yet known

int strip_slots(StripKernel k, const void *kernel) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return 0;
    }
    int slots = g_strip_slots[k][dev].load(std::memory_order_relaxed);
    if (slots > 0) return slots;
    int sms = 0, per_sm = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, 128, 0) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    slots = sms * per_sm;
    g_strip_slots[k][dev].store(slots, std::memory_order_relaxed);
    return slots;
}

// The default height dflt, shortened by two rows at a time (down to lo) while the grid
// fills less than one wave.  For a kernel that keeps the memory system busy, a partly
// filled last wave of many costs little (measured for k_prep at 12 MP), but a grid of
// less than one wave leaves SMs idle.
int fill_rows(int slots, long long blocks_per_rows, int hh, int lo, int dflt) {
    int rows = dflt;
    if (slots <= 0 || blocks_per_rows <= 0 || hh <= 0) return rows;
    while (rows - 2 >= lo && blocks_per_rows * div_up(hh, rows) < slots) rows -= 2;
    return rows;
}

// blocks_per_rows: blocks side by side (columns x frames) per strip of rows
int strip_rows(int slots, long long blocks_per_rows, int hh, int halo, int lo, int hi, int fallback) {
    if (slots <= 0 || blocks_per_rows <= 0 || hh <= 0) return fallback;
    int best = fallback;
    long long best_cost = -1;
    for (int rows = lo; rows <= hi; rows += 2) {
        const long long blocks = blocks_per_rows * div_up(hh, rows);
        const long long cost = ((blocks + slots - 1) / slots) * (rows + halo);
        if (best_cost < 0 || cost < best_cost) { best_cost = cost; best = rows; }
        if (rows >= hh) break;  // one strip covers the frame: longer strips only add rows
    }
    return best;
}

}  // namespace

cudaError_t launch_merge_prep_frames(const uint16_t *burst, const Geom &g, const MergeConsts &c, const MergePlanes &P,
                                     cudaStream_t s, int first_frame) {
    StageRange range("hmfsr merge: 3x3 sums, base statistics and kernel covariance");
    CheckedLaunches checked(s);
    const int nf = g.n - first_frame;
    const int prep_rows = fill_rows(strip_slots(SK_PREP, (const void *)k_prep), (long long)div_up(g.wh, 128) * nf,
                                    g.hh, 8, stage::kPrepStrip);
    k_prep<<<dim3(div_up(g.wh, 128), div_up(g.hh, prep_rows), nf), 128, 0, s>>>(burst, g, c, P.s1, P.base_stats,
                                                                                  P.kern, prep_rows, first_frame);
    if (c.hf_loss > 0.f && g.n > 1)
        k_hf_flag<<<dim3(div_up(g.wh, 128), g.hh), 128, 0, s>>>(burst, P.s1, g, c.hf_loss, P.hf_flag);
    return cudaGetLastError();
}

cudaError_t launch_merge_prep_motion(const float *motion, const Geom &g, const MergeConsts &c, const MergePlanes &P,
                                     cudaStream_t s) {
    StageRange range("hmfsr merge: robustness");
    CheckedLaunches checked(s);
    int nt = g.n * g.ty * g.tx;
    const float2 *mv = reinterpret_cast<const float2 *>(motion);
    k_strength<<<div_up(nt, 128), 128, 0, s>>>(mv, g.n, g.ty, g.tx, c.m_th, c.s1, c.s2, P.s_tile);
    const unsigned char *hf = (c.hf_loss > 0.f && g.n > 1) ? P.hf_flag : nullptr;
    if (g.n > 1) {
        const int slots = hf ? strip_slots(SK_ROB_HF, (const void *)k_rob<true>)
                             : strip_slots(SK_ROB, (const void *)k_rob<false>);
        const int cols = div_up(g.wh, 4 * stage::kRobOut);
        const int rows = strip_rows(slots, (long long)cols * (g.n - 1), g.hh, 4, 8, 256, stage::kRobStrip);
        const dim3 grid(cols, div_up(g.hh, rows), g.n - 1);
        if (hf)
            k_rob<true><<<grid, 128, 0, s>>>(P.s1, P.base_stats, mv, P.s_tile, g, c.t, P.rhat, hf, c.m_th, rows);
        else
            k_rob<false><<<grid, 128, 0, s>>>(P.s1, P.base_stats, mv, P.s_tile, g, c.t, P.rhat, nullptr, c.m_th, rows);
    }
    return cudaGetLastError();
}

cudaError_t launch_merge_prep(const uint16_t *burst, const float *motion, const Geom &g, const MergeConsts &c,
                              const MergePlanes &P, cudaStream_t s) {
    const cudaError_t e = launch_merge_prep_frames(burst, g, c, P, s);
    if (e != cudaSuccess) return e;
    return launch_merge_prep_motion(motion, g, c, P, s);
}

cudaError_t launch_merge_accum(const uint16_t *burst, const float *motion, const Geom &g, const MergePlanes &P,
                               int snum, int sden, float *rgb, float *den, cudaStream_t s) {
    StageRange range("hmfsr merge: accumulation and normalisation");
    CheckedLaunches checked(s);
    int ho = (int)(((long long)g.h * snum) / sden), wo = (int)(((long long)g.w * snum) / sden);
    dim3 grid(div_up(wo, kMergeW), div_up(ho, kMergeH));
    const int ntl = g.ty * g.tx;
    k_geo<<<div_up(g.n * ntl, 128), 128, 0, s>>>(reinterpret_cast<const float2 *>(motion), g.n, ntl, g.ref, 2 * snum,
                                                 P.geo);
    if (den)
        launch_k_merge<true>(grid, s, burst, P.geo, g, P, snum, sden, ho, wo, rgb, den);
    else
        launch_k_merge<false>(grid, s, burst, P.geo, g, P, snum, sden, ho, wo, rgb, nullptr);
    return cudaGetLastError();
}

cudaError_t launch_merge_accum_chunk(const uint16_t *burst, const float *motion, const Geom &g, const MergePlanes &P,
                                     int snum, int sden, float *rgb, float *den, const float *state_in,
                                     float *state_out, bool skip_base, cudaStream_t s) {
    StageRange range("hmfsr merge: accumulation of one chunk of frames");
    CheckedLaunches checked(s);
    const int ho = (int)(((long long)g.h * snum) / sden), wo = (int)(((long long)g.w * snum) / sden);
    const dim3 grid(div_up(wo, kMergeW), div_up(ho, kMergeH));
    const int ntl = g.ty * g.tx;
    k_geo<<<div_up(g.n * ntl, 128), 128, 0, s>>>(reinterpret_cast<const float2 *>(motion), g.n, ntl, g.ref, 2 * snum,
                                                 P.geo);
    stage::ChunkIO io;
    io.state_in = state_in;
    io.state_out = state_out;
    io.skip_base = skip_base ? 1 : 0;
    io.plane = (size_t)ho * wo;
    if (den && !state_out)
        launch_k_merge_chunk<true>(grid, s, burst, P.geo, g, P, snum, sden, ho, wo, rgb, den, io);
    else
        launch_k_merge_chunk<false>(grid, s, burst, P.geo, g, P, snum, sden, ho, wo, rgb, nullptr, io);
    return cudaGetLastError();
}

cudaError_t launch_export_stages(const Geom &g, const MergePlanes &P, float *omega, float *rhat, cudaStream_t s) {
    CheckedLaunches checked(s);
    size_t hw = (size_t)g.hh * g.wh;
    k_export<<<dim3((unsigned)((hw + 255) / 256), g.n), 256, 0, s>>>(P.kern, P.rhat, g.n, g.ref, hw, omega, rhat);
    return cudaGetLastError();
}

}  // namespace hmfsr
