// Tile alignment (Sec. 3.2): the pyramid kernels and the per-burst launch sequence.  The
// searches and the refinement, per tile size, are in align_search.cuh / align_t<T>.cu.
// The per-item bodies live in stages.cuh, shared with the batched persistent kernel.
#include "stages.cuh"

namespace hmfsr {
namespace {

__global__ void k_luma01(const uint16_t *__restrict__ burst, int h, int pitch, int hh, int wh,
                         uint16_t *__restrict__ out0, uint16_t *__restrict__ out1, int lh1, int lw1) {
    stage::luma01(burst, h, pitch, hh, wh, out0, out1, lh1, lw1, blockIdx.x * blockDim.x + threadIdx.x, blockIdx.y,
                  blockIdx.z);
}

// Levels 2 and 3 in one pass: a 16 x 16 block makes a 16 x 16 patch of level 2 (integer
// floor means of 4 x 4 level-1 texels, as down does) in shared memory and, when `l3` is
// set, the 4 x 4 level-3 texels over it (floor means of 4 x 4 level-2 texels).
__global__ void __launch_bounds__(256) k_down23(const uint16_t *__restrict__ l1, int h1, int w1,
                                                uint16_t *__restrict__ l2, int h2, int w2, uint16_t *__restrict__ l3,
                                                int h3, int w3) {
    __shared__ uint32_t patch[16][16];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4, f = blockIdx.z;
    const int x = blockIdx.x * 16 + tx, y = blockIdx.y * 16 + ty;
    uint32_t v = 0;
    if (x < w2 && y < h2) {
        const uint16_t *p = l1 + (size_t)f * h1 * w1 + (size_t)(4 * y) * w1 + 4 * x;
        uint32_t s = 0;
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int i = 0; i < 4; ++i) s += HMFSR_LD(p + (size_t)j * w1 + i);
        v = s / 16u;
        HMFSR_ST(l2 + ((size_t)f * h2 + y) * w2 + x, (uint16_t)v);
    }
    if (l3 == nullptr) return;
    patch[ty][tx] = v;
    __syncthreads();
    if (tx < 4 && ty < 4) {
        const int X = blockIdx.x * 4 + tx, Y = blockIdx.y * 4 + ty;
        if (X < w3 && Y < h3) {  // its 4 x 4 level-2 texels lie inside level 2 (w3 = w2 / 4, h3 = h2 / 4)
            uint32_t s = 0;
#pragma unroll
            for (int j = 0; j < 4; ++j)
#pragma unroll
                for (int i = 0; i < 4; ++i) s += patch[4 * ty + j][4 * tx + i];
            HMFSR_ST(l3 + ((size_t)f * h3 + Y) * w3 + X, (uint16_t)(s / 16u));
        }
    }
}

}  // namespace

cudaError_t launch_align_quadfit(const uint16_t *burst, const Geom &g, const hmfsr_align_params &p,
                                 const AlignLevels &L, float *motion, int32_t *motion_int, cudaStream_t s) {
    StageRange range("hmfsr align with the quadratic-fit subpixel step");
    hmfsr_align_params q = p;
    q.lk_iters = 0;  // the search's vectors; the fit below replaces the Lucas-Kanade step
    cudaError_t e = launch_align(burst, g, q, L, motion, motion_int, s);
    if (e != cudaSuccess) return e;
    switch (p.tile) {
        case 8: return align_quadfit_tiles<4>(g, L, motion, motion_int, s);
        case 16: return align_quadfit_tiles<8>(g, L, motion, motion_int, s);
        case 32: return align_quadfit_tiles<16>(g, L, motion, motion_int, s);
        case 64: return align_quadfit_tiles<32>(g, L, motion, motion_int, s);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_align(const uint16_t *burst, const Geom &g, const hmfsr_align_params &p, const AlignLevels &L,
                         float *motion, int32_t *motion_int, cudaStream_t s) {
    StageRange range("hmfsr align: pyramid, block matching, Lucas-Kanade");
    CheckedLaunches checked(s);
    const int n = g.n;
    // levels 0 and 1 in one pass over the raw burst; the coarser levels from level 1
    const bool two = L.n_levels > 1;
    k_luma01<<<dim3(div_up(g.wh, 4 * 128), div_up(g.hh, 2), n), 128, 0, s>>>(
        burst, g.h, g.pitch, g.hh, g.wh, L.img[0], two ? L.img[1] : nullptr, two ? L.lh[1] : 0, two ? L.lw[1] : 0);
    if (L.n_levels > 2) {
        // levels 2 and 3 (factors 4 and 4) in one pass
        const bool l3 = L.n_levels > 3;
        k_down23<<<dim3(div_up(L.lw[2], 16), div_up(L.lh[2], 16), n), 256, 0, s>>>(
            L.img[1], L.lh[1], L.lw[1], L.img[2], L.lh[2], L.lw[2], l3 ? L.img[3] : nullptr, l3 ? L.lh[3] : 0,
            l3 ? L.lw[3] : 0);
    }
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    switch (p.tile) {
        case 8: return align_search_tiles<4>(g, p, L, motion, motion_int, s);
        case 16: return align_search_tiles<8>(g, p, L, motion, motion_int, s);
        case 32: return align_search_tiles<16>(g, p, L, motion, motion_int, s);
        case 64: return align_search_tiles<32>(g, p, L, motion, motion_int, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace hmfsr
