// Issue-rate probes: the denominators of the accumulation's roofline.  Not part of the
// method.  The accumulation is bound by FP32 and MUFU issue, not by HBM, so its fraction
// of peak needs this GPU's FP32 fused-multiply-add rate and its ex2 rate, measured at
// the clock the GPU runs at, rather than a rate derived from unit counts.
//
// Each thread runs 8 independent dependency chains (enough to cover the pipes' latency
// at 8 warps per scheduler), 16 steps per loop iteration: 128 operations per iteration.
// The result is stored only on a branch no real input takes, so the chains stay live
// without a store per thread.
#include "hmfsr_internal.cuh"

namespace hmfsr {
namespace {

constexpr int kProbeThreads = 256, kProbeChains = 8, kProbeUnroll = 16;

__global__ void __launch_bounds__(kProbeThreads) k_probe_fma(float *sink, int iters, float a, float b) {
    float x[kProbeChains];
#pragma unroll
    for (int c = 0; c < kProbeChains; ++c) x[c] = (float)(threadIdx.x + c) * 1e-3f;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < kProbeUnroll; ++u)
#pragma unroll
            for (int c = 0; c < kProbeChains; ++c) x[c] = fmaf(x[c], a, b);
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kProbeChains; ++c) s += x[c];
    if (s == -1.f) sink[threadIdx.x] = s;  // |x| stays below b / (1 - a): never taken
}

__global__ void __launch_bounds__(kProbeThreads) k_probe_ex2(float *sink, int iters) {
    float x[kProbeChains];
#pragma unroll
    for (int c = 0; c < kProbeChains; ++c) x[c] = 0.5f + (float)(threadIdx.x + c) * 1e-4f;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < kProbeUnroll; ++u)
#pragma unroll
            for (int c = 0; c < kProbeChains; ++c) x[c] = fast_exp2(-x[c]);  // stays in (0.5, 1)
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kProbeChains; ++c) s += x[c];
    if (s == -1.f) sink[threadIdx.x] = s;
}

}  // namespace
}  // namespace hmfsr

using namespace hmfsr;

extern "C" hmfsr_status hmfsr_pipe_probe(int pipe, int blocks, int iters, float *sink_dev, double *lane_ops,
                                         void *stream) {
    if ((pipe != HMFSR_PIPE_FP32_FMA && pipe != HMFSR_PIPE_MUFU_EX2) || blocks < 1 || blocks > (1 << 20) ||
        iters < 1 || iters > (1 << 24) || !sink_dev || (reinterpret_cast<uintptr_t>(sink_dev) & 3))
        return HMFSR_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    if (pipe == HMFSR_PIPE_FP32_FMA)
        k_probe_fma<<<blocks, kProbeThreads, 0, s>>>(sink_dev, iters, 0.999f, 1e-3f);
    else
        k_probe_ex2<<<blocks, kProbeThreads, 0, s>>>(sink_dev, iters);
    if (lane_ops) *lane_ops = (double)blocks * kProbeThreads * (double)iters * (kProbeChains * kProbeUnroll);
    return cudaGetLastError() == cudaSuccess ? HMFSR_OK : HMFSR_ERR_CUDA;
}
