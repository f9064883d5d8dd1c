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
// the same search, then the quadratic-fit subpixel step instead of Lucas-Kanade
cudaError_t launch_align_quadfit(const uint16_t *burst, const Geom &g, const hmfsr_align_params &p,
                                 const AlignLevels &L, float *motion, int32_t *motion_int, cudaStream_t s);

// merge
cudaError_t launch_merge_prep(const uint16_t *burst, const float *motion, const Geom &g, const MergeConsts &c,
                              const MergePlanes &P, cudaStream_t s);
cudaError_t launch_merge_accum(const uint16_t *burst, const float *motion, const Geom &g, const MergePlanes &P,
                               int snum, int sden, float *rgb, float *den, cudaStream_t s);
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
    double *part6;          // [n_bwd_blocks][6] kernel-parameter partial sums
    double *part2;          // [n_rp_blocks][2] (s2, t) partial sums
    unsigned char *sel;     // [n][ty*tx] 1 where the motion prior chose s2
    int n_bwd_blocks, n_rp_blocks;
};
size_t carve_backward(void *ws, const Geom &g, int ho, int wo, size_t fwd_bytes, BwdPlanes *B);
cudaError_t launch_merge_backward(const uint16_t *burst, const float *motion, const Geom &g, const MergeConsts &c,
                                  const MergePlanes &P, const BwdPlanes &B, int snum, int sden, const float *rgb,
                                  const float *lden, const float *grad_rgb, float *grad_params, float *grad_motion,
                                  cudaStream_t s);

}  // namespace hmfsr
