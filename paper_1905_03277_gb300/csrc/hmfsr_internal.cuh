// Internal declarations shared by the hmfsr CUDA translation units (not installed).
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>

#include "hmfsr.h"

namespace hmfsr {

// ---------------------------------------------------------------------------------------
// integer helpers (exact; both operands small)
// ---------------------------------------------------------------------------------------
__host__ __device__ __forceinline__ int floor_div(int a, int b) {  // b > 0
    int q = a / b;
    return (q * b > a) ? q - 1 : q;
}
__host__ __device__ __forceinline__ int clampi(int x, int lo, int hi) { return x < lo ? lo : (x > hi ? hi : x); }
__host__ __device__ __forceinline__ int div_up(int a, int b) { return (a + b - 1) / b; }

// floor(q * v) for a small positive integer q and a float v, exactly: the FP32 product is
// rounded once; when it lands on an integer from above, the exact remainder (fma) says so.
__device__ __forceinline__ int floor_mul(int q, float v) {
    float h = (float)q * v;
    float f = floorf(h);
    if (f == h && fmaf((float)q, v, -h) < 0.0f) f -= 1.0f;
    return (int)f;
}

// 2^x on the SFU (ex2.approx, flush-to-zero): relative error ~2^-22.
// sqrt_rn(x) > t for the FP64 length x = Mx^2 + My^2 (x >= 0 or NaN) and the float t:
// t^2 is exact in FP64, and a correctly rounded square root is monotone with t
// representable, so sqrt_rn(x) > t implies x > t^2; the square root itself (a long FP64
// sequence on this GPU) is then taken only when x > t^2, to settle the rounding at the
// boundary.  The decision is the same as comparing sqrt_rn(x) with t.
__device__ __forceinline__ bool length_exceeds(double x, float t) {
    const double td = (double)t;
    if (td < 0.0) return x == x;  // a length (not NaN) is >= 0 > t
    return x > td * td && __dsqrt_rn(x) > td;
}

__device__ __forceinline__ float fast_exp2(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// 1/x on the SFU (rcp.approx, flush-to-zero): relative error ~2^-23; no range handling.
__device__ __forceinline__ float fast_rcp(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// sqrt on the SFU (sqrt.approx, flush-to-zero): relative error ~2^-23.
__device__ __forceinline__ float fast_sqrt(float x) {
    float y;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// A named NVTX range over the host code that enqueues one stage's launches, so that a
// profiler's timeline groups the kernels by stage (header-only NVTX; without a tool
// attached a push or pop is one indirect call).
struct StageRange {
    explicit StageRange(const char *name) { nvtxRangePushA(name); }
    ~StageRange() { nvtxRangePop(); }
    StageRange(const StageRange &) = delete;
    StageRange &operator=(const StageRange &) = delete;
};

// ---------------------------------------------------------------------------------------
// Checked build (-DHMFSR_CHECKED, a test build of the library, never the default): every
// global load and store of the alignment and merge kernels goes through HMFSR_LDG /
// HMFSR_LD / HMFSR_ST, which check the address against the buffers of the current call
// (the caller's burst, motion, outputs, tables and workspace, as the entry point
// registers them).  An access outside all of them is not made -- a load gives 0, a store
// is dropped -- and the source line of the first such access is recorded in a device
// error word that the host reads back (hmfsr_check_status).  Nothing traps.  Each
// translation unit holds its own copy of the ranges, which its launchers set before
// their launches; calls that register no ranges (n = 0) are not checked.  In the
// default build the macros are plain loads and stores.
// ---------------------------------------------------------------------------------------
constexpr int kCheckMaxRanges = 8;
struct CheckRanges {
    const char *lo[kCheckMaxRanges];
    const char *hi[kCheckMaxRanges];  // one past the last byte
    int n;                            // 0: not checked
    int *err;                         // device word: 0, or the line of the first bad access
};
// the ranges of the current entry-point call on this host thread (api.cu)
const CheckRanges &current_check_ranges();

#ifdef HMFSR_CHECKED
static __constant__ CheckRanges g_check;  // one copy per translation unit

template <typename T>
__device__ __forceinline__ bool check_access(const T *p) {
    if (g_check.n == 0) return true;
    const char *a = reinterpret_cast<const char *>(p);
    for (int i = 0; i < g_check.n; ++i)
        if (a >= g_check.lo[i] && a + sizeof(T) <= g_check.hi[i]) return true;
    return false;
}
__device__ __forceinline__ void check_fail(int site) {
    if (g_check.err) atomicCAS(g_check.err, 0, site);
}
template <typename T>
__device__ __forceinline__ T checked_ldg(const T *p, int site) {
    if (check_access(p)) return __ldg(p);
    check_fail(site);
    return T();
}
template <typename T>
__device__ __forceinline__ T checked_ld(const T *p, int site) {
    if (check_access(p)) return *p;
    check_fail(site);
    return T();
}
template <typename T>
__device__ __forceinline__ void checked_st(T *p, const T &v, int site) {
    if (check_access(p)) *p = v;
    else check_fail(site);
}
#define HMFSR_LDG(p) ::hmfsr::checked_ldg((p), __LINE__)
#define HMFSR_LD(p) ::hmfsr::checked_ld((p), __LINE__)
#define HMFSR_ST(p, v) ::hmfsr::checked_st((p), (v), __LINE__)
// host: for the launches between construction and destruction on stream s, this
// translation unit checks against the current call's ranges; afterwards its launches are
// unchecked again.  Inside stream capture nothing is set (captured launches stay
// unchecked).
struct CheckedLaunches {
    cudaStream_t s;
    bool set = false;
    explicit CheckedLaunches(cudaStream_t s_) : s(s_) {
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        if (cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return;
        const CheckRanges &r = current_check_ranges();
        if (r.n == 0) return;
        set = cudaMemcpyToSymbolAsync(g_check, &r, sizeof(CheckRanges), 0, cudaMemcpyHostToDevice, s) == cudaSuccess;
    }
    ~CheckedLaunches() {
        if (!set) return;
        CheckRanges none = {};
        cudaMemcpyToSymbolAsync(g_check, &none, sizeof(CheckRanges), 0, cudaMemcpyHostToDevice, s);
    }
};
#else
#define HMFSR_LDG(p) __ldg(p)
#define HMFSR_LD(p) (*(p))
#define HMFSR_ST(p, v) ((void)(*(p) = (v)))
struct CheckedLaunches {
    explicit CheckedLaunches(cudaStream_t) {}
};
#endif

// ---------------------------------------------------------------------------------------
// geometry of one burst
// ---------------------------------------------------------------------------------------
struct Geom {
    int n, h, w, pitch, ref, wl;
    int hh, wh;          // half-res size
    int tile, ty, tx;    // motion-field tiles (raw px)
};

// Per-frame merge planes in the workspace (one entry per half-res pixel per frame).
struct MergePlanes {
    uint2 *s1;           // [n][hh*wh] 3x3 guide sums {R | B << 16, G1+G2}
    float4 *base_stats;  // [hh*wh] {max(sum sigma^2, eps), dmd^2 R, G, B} of the base frame
    float4 *kern;        // [n][hh*wh] kernel covariance as {a, delta, ux, uy}: Omega = a I + delta u u^T
    float *rhat;         // [n][hh*wh] final robustness (base grid); unused for the base frame
    float *s_tile;       // [n][ty*tx] robustness scale from the motion prior
    int4 *geo;           // [n][ty*tx] window geometry for the output scale {floor(Q v), Q v - floor(Q v)}
    unsigned char *hf_flag;  // [hh*wh] high-frequency flag of the base texels (when that test is on)
};

// brightness levels of a Monte-Carlo noise table: level i is i WL / (kNoiseLevels - 1)
constexpr int kNoiseLevels = 129, kNoiseTrials = 4096;

struct MergeConsts {
    float k_detail, k_denoise, d_th, d_tr, k_stretch, k_shrink;
    float t, s1, s2, m_th, noise_a, noise_b;
    // nullptr: the closed-form noise statistics; else kNoiseLevels entries
    // {sigma_md^2 red/blue, sigma_md^2 green, d_md^2 red/blue, d_md^2 green}
    const float4 *noise_table;
    // 0: off; else the high-frequency rejection threshold kappa
    float hf_loss;
};

// ---------------------------------------------------------------------------------------
// launchers (return cudaGetLastError() of the launches)
// ---------------------------------------------------------------------------------------
// alignment
struct AlignLevels {
    int n_levels;
    int lh[4], lw[4];          // level sizes
    int lty[4], ltx[4];        // tile grid per level
    uint16_t *img[4];          // [n][lh*lw] per level
    int2 *vec[4];              // [n][lty*ltx] integer vectors per level
};
cudaError_t launch_align(const uint16_t *burst, const Geom &g, const hmfsr_align_params &p, const AlignLevels &L,
                         float *motion, int32_t *motion_int, cudaStream_t s);
// the searches and refinement for tiles of T level texels (one translation unit per T)
template <int T>
cudaError_t align_search_tiles(const Geom &g, const hmfsr_align_params &p, const AlignLevels &L, float *motion,
                               int32_t *motion_int, cudaStream_t s);
template <int T>
cudaError_t align_quadfit_tiles(const Geom &g, const AlignLevels &L, float *motion, int32_t *motion_int,
                                cudaStream_t s);
// the same search, then the quadratic-fit subpixel step instead of Lucas-Kanade
cudaError_t launch_align_quadfit(const uint16_t *burst, const Geom &g, const hmfsr_align_params &p,
                                 const AlignLevels &L, float *motion, int32_t *motion_int, cudaStream_t s);

// merge; launch_merge_prep == launch_merge_prep_frames (the motion-free part: 3x3 sums,
// base statistics, kernel covariances, high-frequency flags) + launch_merge_prep_motion
// (motion strength and robustness)
cudaError_t launch_merge_prep(const uint16_t *burst, const float *motion, const Geom &g, const MergeConsts &c,
                              const MergePlanes &P, cudaStream_t s);
// first_frame: frames first_frame .. n - 1 only (the planes of the earlier ones are kept)
cudaError_t launch_merge_prep_frames(const uint16_t *burst, const Geom &g, const MergeConsts &c, const MergePlanes &P,
                                     cudaStream_t s, int first_frame = 0);
cudaError_t launch_merge_prep_motion(const float *motion, const Geom &g, const MergeConsts &c, const MergePlanes &P,
                                     cudaStream_t s);
cudaError_t launch_merge_accum(const uint16_t *burst, const float *motion, const Geom &g, const MergePlanes &P,
                               int snum, int sden, float *rgb, float *den, cudaStream_t s);
// the accumulation of one chunk of frames of a bounded-memory merge: the running sums
// from state_in (nullptr: start empty) to state_out (nullptr: normalise into rgb / den);
// skip_base: the chunk's burst holds the base frame for the statistics only
cudaError_t launch_merge_accum_chunk(const uint16_t *burst, const float *motion, const Geom &g, const MergePlanes &P,
                                     int snum, int sden, float *rgb, float *den, const float *state_in,
                                     float *state_out, bool skip_base, cudaStream_t s);
cudaError_t launch_export_stages(const Geom &g, const MergePlanes &P, float *omega, float *rhat, cudaStream_t s);

// adjoint of the merge: buffers beyond the forward planes
struct BwdPlanes {
    float4 *shape;          // [n][hh*wh] {A, sqrt(l1_norm), cos 2t, sin 2t}
    float4 *rb;             // [n][hh*wh] {R, dR/dvx, dR/dvy, dR/ds2}
    unsigned char *flags;   // [n][hh*wh] bit 7: R unclamped; bits 0-4: argmin of the 5x5 window
    float *rhbar_tex;       // [n][hh*wh] dL/dRhat on base texels
    float2 *vbar_tex;       // [n][hh*wh] motion contributions through R
    float2 *vbar_pix;       // [n][ho*wo] motion contributions through the weights
    float *rhbar_pix;       // [n][ho*wo] dL/dRhat at output pixels
    float *rhbar_rows;      // [n][ho][wh] dL/dRhat gathered along x (output rows x texel columns)
    double *part6;          // [n_bwd_blocks][6] kernel-parameter partial sums
    double *part2;          // [n_rp_blocks][2] (s2, t) partial sums
    unsigned char *sel;     // [n][ty*tx] 1 where the motion prior chose s2
    int n_bwd_blocks, n_rp_blocks;
};
size_t carve_backward(void *ws, const Geom &g, int ho, int wo, size_t fwd_bytes, BwdPlanes *B);
// the adjoint's four parts (merge_bwd.cu): shape, then robust (after the preparation),
// main (after shape and the preparation), finish (after robust and main)
cudaError_t launch_bwd_shape(const uint16_t *burst, const Geom &g, const BwdPlanes &B, cudaStream_t s);
cudaError_t launch_bwd_robust(const float *motion, const Geom &g, const MergeConsts &c, const MergePlanes &P,
                              const BwdPlanes &B, cudaStream_t s);
cudaError_t launch_bwd_main(const uint16_t *burst, const float *motion, const Geom &g, const MergeConsts &c,
                            const MergePlanes &P, const BwdPlanes &B, int snum, int sden, const float *rgb,
                            const float *lden, const float *grad_rgb, cudaStream_t s);
cudaError_t launch_bwd_finish(const Geom &g, const BwdPlanes &B, int snum, int sden, float *grad_params,
                              float *grad_motion, cudaStream_t s);

}  // namespace hmfsr
