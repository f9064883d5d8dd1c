// Noise-dependent tuning (supplement, "Noise-dependent Tuning" and "Tuning Procedure and
// Parameters"): the base frame's mean brightness and the noise model give an SNR, and the
// kernel parameters and the tile size follow from it.
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

hmfsr_status hmfsr_snr_tuning(double mean, float noise_a, float noise_b, hmfsr_merge_params *mparams,
                              hmfsr_align_params *aparams, double *snr_out) {
    if (!mparams || !aparams || !isfinite(mean) || mean < 0.0 || !isfinite(noise_a) || !isfinite(noise_b) ||
        noise_a < 0.f || noise_b < 0.f)
        return HMFSR_ERR_INVALID_ARG;
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
