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

// One warp per tile of one level: exhaustive integer SSD over offsets |d| <= rad around
// the candidate (parent vector * factor).  Ties: smallest SSD, then smallest |dx|+|dy|,
// then smaller dy, then smaller dx -- encoded in one 64-bit key so that min() decides.
template <int T>
__global__ void k_ssd(const uint16_t *__restrict__ img, int lh, int lw, int lty, int ltx,
                      const int2 *__restrict__ parent, int pty, int ptx, int fct, int rad, int ref,
                      int2 *__restrict__ vec) {
    constexpr int t = T, npx = T * T, nper = (npx + 31) / 32;
    int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    int f = blockIdx.y;
    if (warp >= lty * ltx) return;
    int ty = warp / ltx, tx = warp % ltx;
    int2 *out = vec + (size_t)f * lty * ltx + warp;
    if (f == ref) {
        if (lane == 0) *out = make_int2(0, 0);
        return;
    }
    int cx = 0, cy = 0;
    if (parent) {
        int px = clampi((tx * t + t / 2) / fct / t, 0, ptx - 1);
        int py = clampi((ty * t + t / 2) / fct / t, 0, pty - 1);
        int2 pv = parent[(size_t)f * pty * ptx + (size_t)py * ptx + px];
        cx = pv.x * fct;
        cy = pv.y * fct;
    }
    const uint16_t *R = img + (size_t)ref * lh * lw;
    const uint16_t *A = img + (size_t)f * lh * lw;
    // each lane owns pixels k = lane + 32 m of the tile
    int refv[nper], xs[nper], ys[nper];
#pragma unroll
    for (int m = 0; m < nper; ++m) {
        int k = lane + 32 * m;
        int valid = k < npx;
        int x = tx * t + (valid ? k % t : 0), y = ty * t + (valid ? k / t : 0);
        xs[m] = valid ? x : -100000;
        ys[m] = y;
        refv[m] = valid ? (int)R[(size_t)clampi(y, 0, lh - 1) * lw + clampi(x, 0, lw - 1)] : 0;
    }
    unsigned long long best = ~0ull;
    for (int dy = -rad; dy <= rad; ++dy)
        for (int dx = -rad; dx <= rad; ++dx) {
            long long part = 0;
#pragma unroll
            for (int m = 0; m < nper; ++m) {
                if (xs[m] == -100000) continue;
                int ax = clampi(xs[m] + cx + dx, 0, lw - 1), ay = clampi(ys[m] + cy + dy, 0, lh - 1);
                int d = refv[m] - (int)A[(size_t)ay * lw + ax];
                part += (long long)(d * d);
            }
            long long ssd = warp_sum_ll(part);
            unsigned long long key = ((unsigned long long)ssd << 12) |
                                     ((unsigned long long)(abs(dx) + abs(dy)) << 8) |
                                     ((unsigned long long)(dy + 7) << 4) | (unsigned long long)(dx + 7);
            best = key < best ? key : best;
        }
    if (lane == 0) {
        int bdx = (int)(best & 15ull) - 7, bdy = (int)((best >> 4) & 15ull) - 7;
        *out = make_int2(cx + bdx, cy + bdy);
    }
}

// Lucas-Kanade refinement of one level-0 tile per warp, on I = Lq / 4 (Sec. 3.2).
// Gradients of the base frame by central differences (clamped); H = sum g g^T is summed
// exactly in integers, and the conditioning guard (tr H == 0 or det H <= 1e-9 tr(H)^2) is
// the same IEEE FP64 operation sequence as in any reference implementation; each
// iteration solves H step = -sum g r in FP64 with residuals accumulated in FP32.
template <int T>
__global__ void k_lk(const uint16_t *__restrict__ L0, int lh, int lw, int lty, int ltx,
                     const int2 *__restrict__ vec0, int ref, int iters, float *__restrict__ motion,
                     int32_t *__restrict__ motion_int) {
    int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    int f = blockIdx.y;
    if (warp >= lty * ltx) return;
    int ty = warp / ltx, tx = warp % ltx;
    size_t o = (size_t)f * lty * ltx + warp;
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
    int2 u = vec0[o];
    constexpr int t = T, npx = T * T, nper = (npx + 31) / 32;
    int gxs[nper], gys[nper], pxs[nper], pys[nper], rv[nper];
    long long hxx = 0, hxy = 0, hyy = 0;
#pragma unroll
    for (int m = 0; m < nper; ++m) {
        int k = lane + 32 * m;
        if (k >= npx) { gxs[m] = gys[m] = 0; pxs[m] = pys[m] = 0; rv[m] = 0; continue; }
        int x = clampi(tx * t + k % t, 0, lw - 1), y = clampi(ty * t + k / t, 0, lh - 1);
        int gx = (int)R[(size_t)y * lw + clampi(x + 1, 0, lw - 1)] - (int)R[(size_t)y * lw + clampi(x - 1, 0, lw - 1)];
        int gy = (int)R[(size_t)clampi(y + 1, 0, lh - 1) * lw + x] - (int)R[(size_t)clampi(y - 1, 0, lh - 1) * lw + x];
        gxs[m] = gx; gys[m] = gy; pxs[m] = x; pys[m] = y;
        rv[m] = R[(size_t)y * lw + x];
        hxx += (long long)(gx * gx);
        hxy += (long long)(gx * gy);
        hyy += (long long)(gy * gy);
    }
    hxx = warp_sum_ll(hxx);
    hxy = warp_sum_ll(hxy);
    hyy = warp_sum_ll(hyy);
    double Hxx = (double)hxx, Hxy = (double)hxy, Hyy = (double)hyy;
    double tr = __dadd_rn(Hxx, Hyy);
    double det = __dsub_rn(__dmul_rn(Hxx, Hyy), __dmul_rn(Hxy, Hxy));
    double trsq = __dmul_rn(tr, tr);
    bool skip = (tr == 0.0) || (det <= __dmul_rn(1e-9, trsq));
    float dx = 0.f, dy = 0.f;
    if (!skip) {
        double gxx = Hxx / 64.0, gxy = Hxy / 64.0, gyy = Hyy / 64.0;
        double gdet = gxx * gyy - gxy * gxy;
        for (int it = 0; it < iters; ++it) {
            float fdx = floorf(dx), fdy = floorf(dy);
            float ax = dx - fdx, ay = dy - fdy;
            int ox = u.x + (int)fdx, oy = u.y + (int)fdy;
            float bx = 0.f, by = 0.f;
#pragma unroll
            for (int m = 0; m < nper; ++m) {
                if (lane + 32 * m >= npx) continue;
                int ix = pxs[m] + ox, iy = pys[m] + oy;
                int x0 = clampi(ix, 0, lw - 1), x1 = clampi(ix + 1, 0, lw - 1);
                int y0 = clampi(iy, 0, lh - 1), y1 = clampi(iy + 1, 0, lh - 1);
                float i00 = A[(size_t)y0 * lw + x0], i10 = A[(size_t)y0 * lw + x1];
                float i01 = A[(size_t)y1 * lw + x0], i11 = A[(size_t)y1 * lw + x1];
                float ia = (1.f - ay) * ((1.f - ax) * i00 + ax * i10) + ay * ((1.f - ax) * i01 + ax * i11);
                float r = (ia - (float)rv[m]) * 0.25f;
                bx += (float)gxs[m] * 0.125f * r;
                by += (float)gys[m] * 0.125f * r;
            }
            bx = warp_sum_f(bx);
            by = warp_sum_f(by);
            double sx = -((gyy * bx - gxy * by) / gdet);
            double sy = -((-gxy * bx + gxx * by) / gdet);
            dx = fminf(fmaxf((float)((double)dx + sx), -1.f), 1.f);
            dy = fminf(fmaxf((float)((double)dy + sy), -1.f), 1.f);
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

template <int T>
static void run_search(const Geom &g, const hmfsr_align_params &p, const AlignLevels &L, float *motion,
                       int32_t *motion_int, cudaStream_t s) {
    const int n = g.n;
    for (int l = L.n_levels - 1; l >= 0; --l) {
        int tiles = L.lty[l] * L.ltx[l];
        bool top = (l == L.n_levels - 1);
        k_ssd<T><<<dim3(div_up(tiles * 32, 128), n), 128, 0, s>>>(
            L.img[l], L.lh[l], L.lw[l], L.lty[l], L.ltx[l], top ? nullptr : L.vec[l + 1], top ? 0 : L.lty[l + 1],
            top ? 0 : L.ltx[l + 1], top ? 1 : kFactors[l], p.radius[l], g.ref, L.vec[l]);
    }
    int tiles0 = L.lty[0] * L.ltx[0];
    k_lk<T><<<dim3(div_up(tiles0 * 32, 128), n), 128, 0, s>>>(L.img[0], L.lh[0], L.lw[0], L.lty[0], L.ltx[0],
                                                              L.vec[0], g.ref, p.lk_iters, motion, motion_int);
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
