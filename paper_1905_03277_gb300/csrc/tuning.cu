// The noise model's uses beyond the closed form.  Noise-dependent tuning (supplement,
// "Noise-dependent Tuning" and "Tuning Procedure and Parameters"): the base frame's mean
// brightness and the noise model give an SNR, and the kernel parameters and the tile size
// follow from it.  Monte-Carlo noise statistics (Sec. 5.2.2): the robustness's modelled
// sigma_md^2 and d_md^2 per brightness level, simulated with rounding and clipping.
//
// The mean comes from an exact integer sum of the frame's samples on the GPU
// (hmfsr_frame_sum); the mapping from SNR to parameters is host arithmetic
// (hmfsr_snr_tuning).
#include <math.h>

#include "hmfsr_internal.cuh"

namespace hmfsr {
namespace {

constexpr int kSumThreads = 256, kSumPerThread = 8;

// Sum of every sample of one frame into *sum (zeroed by the caller's stream first).
// Thread t of block (bx, by) reads 8 consecutive samples of the rows by, by + gridDim.y,
// ..., four rows at a time so that four loads are in flight; the partial sums are exact in
// 64 bits and the atomic adds of exact integers commute, so the result does not depend on
// the order.
__device__ __forceinline__ unsigned int sum8(uint4 v) {
    return (v.x & 0xffffu) + (v.x >> 16) + (v.y & 0xffffu) + (v.y >> 16) + (v.z & 0xffffu) + (v.z >> 16) +
           (v.w & 0xffffu) + (v.w >> 16);
}

__global__ void __launch_bounds__(kSumThreads) k_frame_sum(const uint16_t *__restrict__ fr, int h, int w, int pitch,
                                                           unsigned long long *__restrict__ sum) {
    const int x0 = (blockIdx.x * kSumThreads + threadIdx.x) * kSumPerThread;
    const int gy = gridDim.y;
    unsigned long long acc = 0;
    if (x0 < w) {
        const uint16_t *col = fr + x0;
        const bool vec = x0 + kSumPerThread <= w && (pitch & 7) == 0 && (reinterpret_cast<uintptr_t>(col) & 15) == 0;
        if (vec) {
            int y = blockIdx.y;
            for (; y + 3 * gy < h; y += 4 * gy) {
                const uint4 a = __ldg(reinterpret_cast<const uint4 *>(col + (size_t)y * pitch));
                const uint4 b = __ldg(reinterpret_cast<const uint4 *>(col + (size_t)(y + gy) * pitch));
                const uint4 c = __ldg(reinterpret_cast<const uint4 *>(col + (size_t)(y + 2 * gy) * pitch));
                const uint4 d = __ldg(reinterpret_cast<const uint4 *>(col + (size_t)(y + 3 * gy) * pitch));
                acc += (unsigned long long)sum8(a) + sum8(b) + sum8(c) + sum8(d);
            }
            for (; y < h; y += gy) acc += sum8(__ldg(reinterpret_cast<const uint4 *>(col + (size_t)y * pitch)));
        } else {
            for (int y = blockIdx.y; y < h; y += gy)
                for (int i = 0; i < kSumPerThread && x0 + i < w; ++i) acc += __ldg(col + (size_t)y * pitch + i);
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0 && acc) atomicAdd(sum, acc);
}

// ---------------------------------------------------------------------------------------
// Monte-Carlo noise statistics (Sec. 5.2.2: sigma_md and d_md from simulations "for
// different brightness levels", with sensor clipping)
// ---------------------------------------------------------------------------------------
constexpr int kNoiseThreads = 256;

// Philox-4x32-10 (Salmon et al., SC 2011): ten rounds of two 32x32 -> 64-bit products by
// fixed multipliers, the halves recombined with the other counter words and the round
// key; the key is bumped by the Weyl constants between rounds
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        const uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    }
    return c;
}

// normal j of a trial: 12 uniforms (r + 1/2) 2^-32 from three Philox blocks, summed exactly
// (Irwin-Hall), minus 6
__device__ __forceinline__ double noise_normal(int level, int trial, int j) {
    unsigned long long s = 0;
#pragma unroll
    for (int b = 0; b < 3; ++b) {
        const uint4 o = philox4x32_10(make_uint4((uint32_t)(3 * j + b), (uint32_t)trial, (uint32_t)level, 0u),
                                      0x19050327u, 0x5EED0001u);
        s += (unsigned long long)o.x + o.y + o.z + o.w;
    }
    return __dadd_rn(__dmul_rn(__dadd_rn((double)s, 6.0), 1.0 / 4294967296.0), -6.0);
}

// one raw sample of a constant patch: rounded to a whole DN and clipped to [0, WL], in
// FP64 with the same operation sequence as a CPU restatement, so every decision agrees
__device__ __forceinline__ double noise_sample(double x, double sigma, double wl, int level, int trial, int j) {
    const double v = floor(__dadd_rn(__dadd_rn(x, __dmul_rn(sigma, noise_normal(level, trial, j))), 0.5));
    return fmin(fmax(v, 0.0), wl);
}

// One block per brightness level; each thread takes every kNoiseThreads-th trial.  A
// trial draws two independent 3x3 patches of guide pixels (red/blue: one sample; green:
// the mean of two) and adds {population variance of patch 1, red/blue and green;
// squared difference of the two patch means, red/blue and green}; the block's FP64 sums
// become the level's trial means.
__global__ void __launch_bounds__(kNoiseThreads) k_noise_table(float noise_a, float noise_b, int wl,
                                                               float4 *__restrict__ table) {
    __shared__ double red[4][kNoiseThreads];
    const int level = blockIdx.x;
    const double x = __ddiv_rn(__dmul_rn((double)level, (double)wl), (double)(kNoiseLevels - 1));
    const double var = __dadd_rn(__dmul_rn((double)noise_a, x), (double)noise_b);
    const double sigma = var > 0.0 ? __dsqrt_rn(var) : 0.0;
    const double dwl = (double)wl;
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    for (int t = threadIdx.x; t < kNoiseTrials; t += kNoiseThreads) {
        double mean[2][2], var1[2];
#pragma unroll
        for (int ch = 0; ch < 2; ++ch) {
            double v1[9];
#pragma unroll 1
            for (int q = 0; q < 2; ++q) {
                double s = 0.0;
#pragma unroll 1
                for (int k = 0; k < 9; ++k) {
                    double v;
                    if (ch == 0) {
                        v = noise_sample(x, sigma, dwl, level, t, 27 * q + k);
                    } else {
                        v = __dmul_rn(0.5, __dadd_rn(noise_sample(x, sigma, dwl, level, t, 27 * q + 9 + 2 * k),
                                                     noise_sample(x, sigma, dwl, level, t, 27 * q + 10 + 2 * k)));
                    }
                    if (q == 0) v1[k] = v;
                    s = __dadd_rn(s, v);
                }
                mean[ch][q] = __ddiv_rn(s, 9.0);
            }
            double ss = 0.0;
#pragma unroll
            for (int k = 0; k < 9; ++k) {
                const double d = __dadd_rn(v1[k], -mean[ch][0]);
                ss = __dadd_rn(ss, __dmul_rn(d, d));
            }
            var1[ch] = __ddiv_rn(ss, 9.0);
        }
        acc[0] = __dadd_rn(acc[0], var1[0]);
        acc[1] = __dadd_rn(acc[1], var1[1]);
        const double d0 = __dadd_rn(mean[0][0], -mean[0][1]), d1 = __dadd_rn(mean[1][0], -mean[1][1]);
        acc[2] = __dadd_rn(acc[2], __dmul_rn(d0, d0));
        acc[3] = __dadd_rn(acc[3], __dmul_rn(d1, d1));
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) red[k][threadIdx.x] = acc[k];
    __syncthreads();
    for (int m = kNoiseThreads / 2; m > 0; m >>= 1) {
        if (threadIdx.x < m)
#pragma unroll
            for (int k = 0; k < 4; ++k) red[k][threadIdx.x] += red[k][threadIdx.x + m];
        __syncthreads();
    }
    if (threadIdx.x == 0)
        table[level] = make_float4((float)(red[0][0] / kNoiseTrials), (float)(red[1][0] / kNoiseTrials),
                                   (float)(red[2][0] / kNoiseTrials), (float)(red[3][0] / kNoiseTrials));
}

// piecewise-linear parameter between its value at SNR 6 (low) and at SNR 30 (high)
double lerp_snr(double lo, double hi, double snr) {
    const double t = fmin(fmax((snr - 6.0) / 24.0, 0.0), 1.0);
    return (1.0 - t) * lo + t * hi;  // both ends exact
}

}  // namespace
}  // namespace hmfsr

using namespace hmfsr;

extern "C" {

hmfsr_status hmfsr_frame_sum(const uint16_t *burst_dev, const hmfsr_burst_desc *desc, int frame,
                             unsigned long long *sum_dev, void *stream) {
    if (!desc || !burst_dev || !sum_dev || frame < 0 || frame >= desc->n_frames || desc->height < 1 ||
        desc->width < 1 || desc->pitch_elems < desc->width || (reinterpret_cast<uintptr_t>(sum_dev) & 7))
        return HMFSR_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    if (cudaMemsetAsync(sum_dev, 0, sizeof(unsigned long long), s) != cudaSuccess) return HMFSR_ERR_CUDA;
    const int gx = div_up(desc->width, kSumThreads * kSumPerThread);
    // about 4 blocks per SM in all, each thread over ~h / gy rows
    const int gy = max(1, min(div_up(desc->height, 4), (152 * 4) / gx));
    const uint16_t *fr = burst_dev + (size_t)frame * desc->height * desc->pitch_elems;
    k_frame_sum<<<dim3(gx, gy), kSumThreads, 0, s>>>(fr, desc->height, desc->width, desc->pitch_elems, sum_dev);
    return cudaGetLastError() == cudaSuccess ? HMFSR_OK : HMFSR_ERR_CUDA;
}

hmfsr_status hmfsr_noise_table(float noise_a, float noise_b, int white_level, float *table_dev, void *stream) {
    if (!table_dev || (reinterpret_cast<uintptr_t>(table_dev) & 15) || !isfinite(noise_a) || !isfinite(noise_b) ||
        noise_a < 0.f || noise_b < 0.f || white_level < 1 || white_level > 65535)
        return HMFSR_ERR_INVALID_ARG;
    k_noise_table<<<kNoiseLevels, kNoiseThreads, 0, (cudaStream_t)stream>>>(noise_a, noise_b, white_level,
                                                                          reinterpret_cast<float4 *>(table_dev));
    return cudaGetLastError() == cudaSuccess ? HMFSR_OK : HMFSR_ERR_CUDA;
}

hmfsr_status hmfsr_snr_tuning(uint64_t sample_sum, uint64_t sample_count, float noise_a, float noise_b,
                              hmfsr_merge_params *mparams, hmfsr_align_params *aparams, double *snr_out) {
    // both below 2^53: exact as doubles, so the mean is the correctly rounded quotient
    if (!mparams || !aparams || sample_count == 0 || sample_count >= (1ull << 53) || sample_sum >= (1ull << 53) ||
        !isfinite(noise_a) || !isfinite(noise_b) || noise_a < 0.f || noise_b < 0.f)
        return HMFSR_ERR_INVALID_ARG;
    const double mean = (double)sample_sum / (double)sample_count;
    // SNR of one raw sample of a single frame at the mean brightness
    const double var = (double)noise_a * mean + (double)noise_b;
    const double snr = var > 0.0 ? mean / sqrt(var) : INFINITY;
    const double snr_c = isinf(snr) ? 30.0 : snr;
    // the tile grows from 16 px to 64 px only in very low light: the lowest third of the
    // SNR range, split in two
    const int tile = snr_c < 10.0 ? 64 : (snr_c < 14.0 ? 32 : 16);
    mparams->k_detail = (float)lerp_snr(0.33, 0.25, snr_c);
    mparams->k_denoise = (float)lerp_snr(5.0, 3.0, snr_c);
    mparams->d_th = (float)lerp_snr(0.010, 0.001, snr_c);
    mparams->d_tr = (float)lerp_snr(0.020, 0.006, snr_c);
    mparams->k_stretch = 4.f;
    mparams->k_shrink = 2.f;
    mparams->t = 0.12f;
    mparams->s1 = 12.f;
    mparams->s2 = 2.f;
    mparams->m_th = 0.8f;
    mparams->noise_a = noise_a;
    mparams->noise_b = noise_b;
    mparams->tile = tile;
    aparams->tile = tile;
    aparams->n_levels = 4;
    aparams->radius[0] = 1;
    aparams->radius[1] = aparams->radius[2] = aparams->radius[3] = 4;
    aparams->lk_iters = 3;
    if (snr_out) *snr_out = snr;
    return HMFSR_OK;
}

}  // extern "C"
