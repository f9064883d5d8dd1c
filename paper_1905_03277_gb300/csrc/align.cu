// Tile alignment (Sec. 3.2): pyramid block matching with an exact integer SSD search,
// then Lucas-Kanade refinement.  One warp per tile; SSD and normal-equation sums are
// warp-shuffle reductions.
#include "hmfsr_internal.cuh"

namespace hmfsr {
namespace {


// Level 0 = half-res luminance Lq: sum of the four Bayer samples of each quad (Sec. 5.1.2).
__global__ void k_luma0(const uint16_t *__restrict__ burst, int h, int w, int pitch, int hh, int wh,
                        uint16_t *__restrict__ out) {
    int u = blockIdx.x * blockDim.x + threadIdx.x;
    int v = blockIdx.y;
    int f = blockIdx.z;
    if (u >= wh) return;
    const uint16_t *r0 = burst + ((size_t)f * h + 2 * v) * pitch + 2 * u;
    uint32_t a = __ldg(reinterpret_cast<const uint32_t *>(r0));
    uint32_t b = __ldg(reinterpret_cast<const uint32_t *>(r0 + pitch));
    uint32_t s = (a & 0xffffu) + (a >> 16) + (b & 0xffffu) + (b >> 16);
    out[((size_t)f * hh + v) * wh + u] = (uint16_t)s;
}

// Next level: integer floor mean of f x f blocks.
__global__ void k_down(const uint16_t *__restrict__ src, int sh, int sw, uint16_t *__restrict__ dst, int dh, int dw,
                       int fct) {
    int x = blockIdx.x * blockDim.x + threadIdx.x;
    int y = blockIdx.y;
    int f = blockIdx.z;
    if (x >= dw) return;
    const uint16_t *p = src + (size_t)f * sh * sw + (size_t)(y * fct) * sw + x * fct;
    uint32_t s = 0;
    for (int j = 0; j < fct; ++j)
        for (int i = 0; i < fct; ++i) s += p[(size_t)j * sw + i];
    dst[((size_t)f * dh + y) * dw + x] = (uint16_t)(s / (uint32_t)(fct * fct));
}

constexpr int kMaxRad = 7;

__device__ __forceinline__ long long warp_sum_ll(long long v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ float warp_sum_f(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// One thread per tile of one level: exhaustive integer SSD over offsets |d| <= RAD
// around the candidate (the parent's vector times the level factor).  For each dy the
// thread streams the tile's rows (L1-cached reads, clamped at the border) and keeps the
// 2 RAD + 1 candidate sums of that row of offsets in registers.  Ties: smallest SSD,
// then smallest |dx| + |dy|, then smaller dy, then smaller dx -- one 64-bit key whose
// minimum decides.
template <int T, int RAD>
__global__ void __launch_bounds__(64) k_ssd(const uint16_t *__restrict__ img, int lh, int lw, int lty, int ltx,
                                            const int2 *__restrict__ parent, int pty, int ptx, int fsh, int ref,
                                            int2 *__restrict__ vec) {
    constexpr int kW = 2 * RAD + 1;
    const int tile = blockIdx.x * blockDim.x + threadIdx.x;
    const int f = blockIdx.y;
    if (tile >= lty * ltx) return;
    const int ty = tile / ltx, tx = tile - ty * ltx;
    int2 *out = vec + (size_t)f * lty * ltx + tile;
    if (f == ref) {
        *out = make_int2(0, 0);
        return;
    }
    int cx = 0, cy = 0;
    if (parent) {  // level factor 1 << fsh
        const int px = min(((tx * T + T / 2) >> fsh) / T, ptx - 1);
        const int py = min(((ty * T + T / 2) >> fsh) / T, pty - 1);
        const int2 pv = __ldg(parent + (size_t)f * pty * ptx + (size_t)py * ptx + px);
        cx = pv.x << fsh;
        cy = pv.y << fsh;
    }
    const uint16_t *R = img + (size_t)ref * lh * lw;
    const uint16_t *A = img + (size_t)f * lh * lw;
    const int x0 = tx * T, y0 = ty * T;
    unsigned long long best = ~0ull;
    for (int dy = -RAD; dy <= RAD; ++dy) {
        unsigned long long acc[kW];
#pragma unroll
        for (int k = 0; k < kW; ++k) acc[k] = 0;
        for (int j = 0; j < T; ++j) {
            const uint16_t *rrow = R + (size_t)min(y0 + j, lh - 1) * lw;
            const uint16_t *arow = A + (size_t)clampi(y0 + j + cy + dy, 0, lh - 1) * lw;
            int rv[T], av[T + 2 * RAD];
#pragma unroll
            for (int i = 0; i < T; ++i) rv[i] = __ldg(rrow + min(x0 + i, lw - 1));
#pragma unroll
            for (int i = 0; i < T + 2 * RAD; ++i) av[i] = __ldg(arow + clampi(x0 + cx - RAD + i, 0, lw - 1));
#pragma unroll
            for (int k = 0; k < kW; ++k) {
#pragma unroll
                for (int i0 = 0; i0 < T; i0 += 8) {
                    unsigned int part = 0;  // 8 squared 14-bit differences fit 32 bits
#pragma unroll
                    for (int i = i0; i < i0 + 8 && i < T; ++i) {
                        const int d = rv[i] - av[i + k];
                        part += (unsigned int)(d * d);
                    }
                    acc[k] += part;
                }
            }
        }
#pragma unroll
        for (int k = 0; k < kW; ++k) {
            const int dx = k - RAD;
            const unsigned long long key = (acc[k] << 12) | ((unsigned long long)(abs(dx) + abs(dy)) << 8) |
                                           ((unsigned long long)(dy + 7) << 4) | (unsigned long long)(dx + 7);
            best = key < best ? key : best;
        }
    }
    const int bdx = (int)(best & 15ull) - 7, bdy = (int)((best >> 4) & 15ull) - 7;
    *out = make_int2(cx + bdx, cy + bdy);
}

// Lucas-Kanade refinement (Sec. 3.2) of one level-0 tile per warp, on I = Lq / 4.  Each
// lane owns pixels lane + 32 m of the tile.  Gradients of the base frame by central
// differences around the clamped pixel; H = sum g g^T is summed exactly in integers, so
// the conditioning guard (tr H == 0 or det H <= 1e-9 tr(H)^2) is an exact 128-bit integer
// test; each iteration accumulates sum g r in FP32 (warp shuffles) and solves the 2x2
// system.
template <int T>
__global__ void k_lk(const uint16_t *__restrict__ L0, int lh, int lw, int lty, int ltx,
                     const int2 *__restrict__ vec0, int ref, int iters, float *__restrict__ motion,
                     int32_t *__restrict__ motion_int) {
    constexpr int t = T, npx = T * T, nper = (npx + 31) / 32;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    const int f = blockIdx.y;
    if (warp >= lty * ltx) return;
    const int ty = warp / ltx, tx = warp % ltx;
    const size_t o = (size_t)f * lty * ltx + warp;
    if (f == ref) {
        if (lane == 0) {
            motion[2 * o] = 0.f;
            motion[2 * o + 1] = 0.f;
            if (motion_int) { motion_int[2 * o] = 0; motion_int[2 * o + 1] = 0; }
        }
        return;
    }
    const uint16_t *R = L0 + (size_t)ref * lh * lw;
    const uint16_t *A = L0 + (size_t)f * lh * lw;
    const int2 u = vec0[o];
    int gxs[nper], gys[nper], pxs[nper], pys[nper], rv[nper];
    long long hxx = 0, hxy = 0, hyy = 0;
#pragma unroll
    for (int m = 0; m < nper; ++m) {
        const int k = lane + 32 * m;
        if (k >= npx) { gxs[m] = gys[m] = 0; pxs[m] = pys[m] = 0; rv[m] = 0; continue; }
        const int x = min(tx * t + k % t, lw - 1), y = min(ty * t + k / t, lh - 1);
        const uint16_t *row = R + (size_t)y * lw;
        const int gx = (int)__ldg(row + min(x + 1, lw - 1)) - (int)__ldg(row + max(x - 1, 0));
        const int gy = (int)__ldg(R + (size_t)min(y + 1, lh - 1) * lw + x) - (int)__ldg(R + (size_t)max(y - 1, 0) * lw + x);
        gxs[m] = gx; gys[m] = gy; pxs[m] = x; pys[m] = y;
        rv[m] = __ldg(row + x);
        hxx += (long long)(gx * gx);
        hxy += (long long)(gx * gy);
        hyy += (long long)(gy * gy);
    }
    hxx = warp_sum_ll(hxx);
    hxy = warp_sum_ll(hxy);
    hyy = warp_sum_ll(hyy);
    // conditioning guard, exact: skip when tr H == 0 or 10^9 det H <= tr(H)^2
    const __int128 det_i = (__int128)hxx * hyy - (__int128)hxy * hxy;
    const __int128 tr_i = (__int128)hxx + hyy;
    const bool skip = (tr_i == 0) || ((__int128)1000000000 * det_i <= tr_i * tr_i);
    float dx = 0.f, dy = 0.f;
    if (!skip) {
        // H in units of g = (Lq difference) / 8 is H_int / 64
        const float Hxx = (float)hxx, Hxy = (float)hxy, Hyy = (float)hyy;
        const float inv = 64.f / fmaf(Hxx, Hyy, -Hxy * Hxy);
        for (int it = 0; it < iters; ++it) {
            const float fdx = floorf(dx), fdy = floorf(dy);
            const float ax = dx - fdx, ay = dy - fdy;
            const int ox = u.x + (int)fdx, oy = u.y + (int)fdy;
            float bx = 0.f, by = 0.f;
#pragma unroll
            for (int m = 0; m < nper; ++m) {
                if (lane + 32 * m >= npx) continue;
                const int ix = pxs[m] + ox, iy = pys[m] + oy;
                const int x0 = clampi(ix, 0, lw - 1), x1 = clampi(ix + 1, 0, lw - 1);
                const uint16_t *a0 = A + (size_t)clampi(iy, 0, lh - 1) * lw;
                const uint16_t *a1 = A + (size_t)clampi(iy + 1, 0, lh - 1) * lw;
                const float i00 = __ldg(a0 + x0), i10 = __ldg(a0 + x1), i01 = __ldg(a1 + x0), i11 = __ldg(a1 + x1);
                const float ia = (1.f - ay) * ((1.f - ax) * i00 + ax * i10) + ay * ((1.f - ax) * i01 + ax * i11);
                const float r = (ia - (float)rv[m]) * 0.25f;
                bx = fmaf((float)gxs[m] * 0.125f, r, bx);
                by = fmaf((float)gys[m] * 0.125f, r, by);
            }
            bx = warp_sum_f(bx);
            by = warp_sum_f(by);
            const float sx = -(Hyy * bx - Hxy * by) * inv;
            const float sy = -(Hxx * by - Hxy * bx) * inv;
            dx = fminf(fmaxf(dx + sx, -1.f), 1.f);
            dy = fminf(fmaxf(dy + sy, -1.f), 1.f);
        }
    }
    if (lane == 0) {
        motion[2 * o] = 2.f * ((float)u.x + dx);
        motion[2 * o + 1] = 2.f * ((float)u.y + dy);
        if (motion_int) { motion_int[2 * o] = u.x; motion_int[2 * o + 1] = u.y; }
    }
}

}  // namespace

static const int kFactors[3] = {2, 4, 4};

template <int T, int RAD>
static void launch_ssd(const AlignLevels &L, int l, int n, int ref, int fsh, bool top, cudaStream_t s) {
    const int tiles = L.lty[l] * L.ltx[l];
    k_ssd<T, RAD><<<dim3(div_up(tiles, 64), n), 64, 0, s>>>(
        L.img[l], L.lh[l], L.lw[l], L.lty[l], L.ltx[l], top ? nullptr : L.vec[l + 1], top ? 0 : L.lty[l + 1],
        top ? 0 : L.ltx[l + 1], fsh, ref, L.vec[l]);
}

template <int T>
static void run_search(const Geom &g, const hmfsr_align_params &p, const AlignLevels &L, float *motion,
                       int32_t *motion_int, cudaStream_t s) {
    static const int kShift[3] = {1, 2, 2};  // log2 of the factors 2, 4, 4
    const int n = g.n;
    for (int l = L.n_levels - 1; l >= 0; --l) {
        const bool top = (l == L.n_levels - 1);
        const int fsh = top ? 0 : kShift[l];
        switch (p.radius[l]) {
            case 0: launch_ssd<T, 0>(L, l, n, g.ref, fsh, top, s); break;
            case 1: launch_ssd<T, 1>(L, l, n, g.ref, fsh, top, s); break;
            case 2: launch_ssd<T, 2>(L, l, n, g.ref, fsh, top, s); break;
            case 3: launch_ssd<T, 3>(L, l, n, g.ref, fsh, top, s); break;
            case 4: launch_ssd<T, 4>(L, l, n, g.ref, fsh, top, s); break;
            case 5: launch_ssd<T, 5>(L, l, n, g.ref, fsh, top, s); break;
            case 6: launch_ssd<T, 6>(L, l, n, g.ref, fsh, top, s); break;
            default: launch_ssd<T, kMaxRad>(L, l, n, g.ref, fsh, top, s); break;
        }
    }
    const int tiles0 = L.lty[0] * L.ltx[0];
    k_lk<T><<<dim3(div_up(tiles0 * 32, 128), n), 128, 0, s>>>(L.img[0], L.lh[0], L.lw[0], L.lty[0], L.ltx[0], L.vec[0],
                                                       g.ref, p.lk_iters, motion, motion_int);
}

cudaError_t launch_align(const uint16_t *burst, const Geom &g, const hmfsr_align_params &p, const AlignLevels &L,
                         float *motion, int32_t *motion_int, cudaStream_t s) {
    const int n = g.n;
    k_luma0<<<dim3(div_up(g.wh, 128), g.hh, n), 128, 0, s>>>(burst, g.h, g.w, g.pitch, g.hh, g.wh, L.img[0]);
    for (int l = 1; l < L.n_levels; ++l)
        k_down<<<dim3(div_up(L.lw[l], 128), L.lh[l], n), 128, 0, s>>>(L.img[l - 1], L.lh[l - 1], L.lw[l - 1],
                                                                       L.img[l], L.lh[l], L.lw[l], kFactors[l - 1]);
    switch (p.tile) {
        case 8: run_search<4>(g, p, L, motion, motion_int, s); break;
        case 16: run_search<8>(g, p, L, motion, motion_int, s); break;
        case 32: run_search<16>(g, p, L, motion, motion_int, s); break;
        case 64: run_search<32>(g, p, L, motion, motion_int, s); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace hmfsr
