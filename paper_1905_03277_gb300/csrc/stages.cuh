// Per-item bodies of the alignment and merge-preparation stages, shared by the
// per-burst kernels and the batched persistent kernel so that both run exactly the same
// arithmetic.  Each function handles the work of one thread, or where stated one warp,
// given its decoded indices.  The accumulation is in accumulate.cuh.
#pragma once

#include "hmfsr_internal.cuh"

namespace hmfsr {
namespace stage {

constexpr float kHalfLog2e = 0.72134752044448170368f;  // log2(e) / 2
constexpr float kBig = 1.0e30f;

// ======================================================================================
// alignment (Sec. 3.2)
// ======================================================================================
// Level 0 = half-res luminance Lq: sum of the four Bayer samples of each quad (Sec. 5.1.2).
// One thread makes 4 consecutive texels: two 16-byte loads and one 8-byte store where the
// rows allow it, else 4 scalar quads.
__device__ __forceinline__ void luma0(const uint16_t *__restrict__ burst, int h, int pitch, int hh, int wh,
                                      uint16_t *__restrict__ out, int u4, int v, int f) {
    const int u = 4 * u4;
    if (u >= wh) return;
    const uint16_t *r0 = burst + ((size_t)f * h + 2 * v) * pitch + 2 * u;
    uint16_t *o = out + ((size_t)f * hh + v) * wh + u;
    if (u + 4 <= wh && ((reinterpret_cast<uintptr_t>(r0) | reinterpret_cast<uintptr_t>(r0 + pitch)) & 15) == 0 &&
        (reinterpret_cast<uintptr_t>(o) & 7) == 0) {
        const uint4 a = HMFSR_LDG(reinterpret_cast<const uint4 *>(r0));
        const uint4 b = HMFSR_LDG(reinterpret_cast<const uint4 *>(r0 + pitch));
        const uint32_t s0 = (a.x & 0xffffu) + (a.x >> 16) + (b.x & 0xffffu) + (b.x >> 16);
        const uint32_t s1 = (a.y & 0xffffu) + (a.y >> 16) + (b.y & 0xffffu) + (b.y >> 16);
        const uint32_t s2 = (a.z & 0xffffu) + (a.z >> 16) + (b.z & 0xffffu) + (b.z >> 16);
        const uint32_t s3 = (a.w & 0xffffu) + (a.w >> 16) + (b.w & 0xffffu) + (b.w >> 16);
        HMFSR_ST(reinterpret_cast<uint2 *>(o), make_uint2(s0 | (s1 << 16), s2 | (s3 << 16)));
        return;
    }
    for (int i = 0; i < 4 && u + i < wh; ++i) {
        const uint32_t a = HMFSR_LDG(reinterpret_cast<const uint32_t *>(r0 + 2 * i));
        const uint32_t b = HMFSR_LDG(reinterpret_cast<const uint32_t *>(r0 + pitch + 2 * i));
        HMFSR_ST(o + i, (uint16_t)((a & 0xffffu) + (a >> 16) + (b & 0xffffu) + (b >> 16)));
    }
}

// Levels 0 and 1 together: one thread makes 4 texels in each of the level-0 rows 2 y and
// 2 y + 1 (as luma0 does) and, from those 8, the 2 level-1 texels they cover (integer floor
// mean of 2 x 2, as down with factor 2 does), so the first reduction needs no second pass
// over level 0.  out1 = nullptr: level 0 only.
__device__ __forceinline__ void luma01(const uint16_t *__restrict__ burst, int h, int pitch, int hh, int wh,
                                       uint16_t *__restrict__ out0, uint16_t *__restrict__ out1, int lh1, int lw1,
                                       int u4, int y, int f) {
    const int u = 4 * u4;
    if (u >= wh) return;
    uint32_t sq[2][4];
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        const int v = 2 * y + r;
#pragma unroll
        for (int i = 0; i < 4; ++i) sq[r][i] = 0u;
        if (v >= hh) continue;
        const uint16_t *r0 = burst + ((size_t)f * h + 2 * v) * pitch + 2 * u;
        uint16_t *o = out0 + ((size_t)f * hh + v) * wh + u;
        if (u + 4 <= wh && ((reinterpret_cast<uintptr_t>(r0) | reinterpret_cast<uintptr_t>(r0 + pitch)) & 15) == 0 &&
            (reinterpret_cast<uintptr_t>(o) & 7) == 0) {
            const uint4 a = HMFSR_LDG(reinterpret_cast<const uint4 *>(r0));
            const uint4 b = HMFSR_LDG(reinterpret_cast<const uint4 *>(r0 + pitch));
            sq[r][0] = (a.x & 0xffffu) + (a.x >> 16) + (b.x & 0xffffu) + (b.x >> 16);
            sq[r][1] = (a.y & 0xffffu) + (a.y >> 16) + (b.y & 0xffffu) + (b.y >> 16);
            sq[r][2] = (a.z & 0xffffu) + (a.z >> 16) + (b.z & 0xffffu) + (b.z >> 16);
            sq[r][3] = (a.w & 0xffffu) + (a.w >> 16) + (b.w & 0xffffu) + (b.w >> 16);
            HMFSR_ST(reinterpret_cast<uint2 *>(o), make_uint2(sq[r][0] | (sq[r][1] << 16), sq[r][2] | (sq[r][3] << 16)));
        } else {
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                if (u + i >= wh) break;
                const uint32_t a = HMFSR_LDG(reinterpret_cast<const uint32_t *>(r0 + 2 * i));
                const uint32_t b = HMFSR_LDG(reinterpret_cast<const uint32_t *>(r0 + pitch + 2 * i));
                sq[r][i] = (a & 0xffffu) + (a >> 16) + (b & 0xffffu) + (b >> 16);
                HMFSR_ST(o + i, (uint16_t)sq[r][i]);
            }
        }
    }
    if (out1 == nullptr || y >= lh1) return;
    uint16_t *o1 = out1 + ((size_t)f * lh1 + y) * lw1;
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const int x = u / 2 + k;  // level-1 texel over level-0 columns 2 x, 2 x + 1
        if (x < lw1) HMFSR_ST(o1 + x, (uint16_t)((sq[0][2 * k] + sq[0][2 * k + 1] + sq[1][2 * k] + sq[1][2 * k + 1]) / 4u));
    }
}

// Next level: integer floor mean of f x f blocks.
__device__ __forceinline__ void down(const uint16_t *__restrict__ src, int sh, int sw, uint16_t *__restrict__ dst,
                                     int dh, int dw, int fct, int x, int y, int f) {
    if (x >= dw) return;
    const uint16_t *p = src + (size_t)f * sh * sw + (size_t)(y * fct) * sw + x * fct;
    uint32_t s = 0;
    for (int j = 0; j < fct; ++j)
        for (int i = 0; i < fct; ++i) s += HMFSR_LD(p + (size_t)j * sw + i);
    HMFSR_ST(dst + ((size_t)f * dh + y) * dw + x, (uint16_t)(s / (uint32_t)(fct * fct)));
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

// Squared differences of one tile row against one candidate row, exactly, summed PART at
// a time in 32 bits before the 64-bit total: with level values v <= vmax, PART terms fit
// 32 bits while PART vmax^2 < 2^32 (PART = 4 for vmax < 2^15, any white level up to
// 7281; PART = 16 for vmax < 2^14, white levels up to 4095).
template <int T, int PART = 4>
__device__ __forceinline__ unsigned long long row_ssd(const int *rv, const int *av) {
    unsigned long long acc = 0;
#pragma unroll
    for (int i0 = 0; i0 < T; i0 += PART) {
        unsigned int part = 0;
#pragma unroll
        for (int i = i0; i < i0 + PART && i < T; ++i) {
            const int d = rv[i] - av[i];
            part += (unsigned int)(d * d);
        }
        acc += part;
    }
    return acc;
}

// One tile row's squared differences as a 32-bit partial (T <= PART terms).
template <int T>
__device__ __forceinline__ unsigned int row_sq32(const int *rv, const int *av) {
    unsigned int part = 0;
#pragma unroll
    for (int i = 0; i < T; ++i) {
        const int d = rv[i] - av[i];
        part += (unsigned int)(d * d);
    }
    return part;
}

// Exact SSD accumulation over the rows of a tile for one candidate: rows are summed into a
// 32-bit partial PART / T rows at a time (T <= PART), else split PART terms at a time.
template <int T, int PART>
struct SsdAcc {
    static constexpr int kRows = PART >= T ? PART / T : 1;  // rows per 32-bit partial
    unsigned long long total = 0;
    unsigned int part = 0;
    // add row j (0 <= j < T) of the tile
    __device__ __forceinline__ void add(const int *rv, const int *av, int j) {
        if constexpr (PART >= T) {
            part += row_sq32<T>(rv, av);
            if ((j + 1) % kRows == 0 || j == T - 1) {
                total += part;
                part = 0;
            }
        } else {
            total += row_ssd<T, PART>(rv, av);
        }
    }
};

// The block-matching key: smallest SSD, then smallest |dx| + |dy|, then smaller dy, then
// smaller dx -- one 64-bit key whose minimum decides.
__device__ __forceinline__ unsigned long long ssd_key(unsigned long long ssd, int dx, int dy) {
    return (ssd << 12) | ((unsigned long long)(abs(dx) + abs(dy)) << 8) | ((unsigned long long)(dy + 7) << 4) |
           (unsigned long long)(dx + 7);
}

// candidate centre of a tile: the parent level's vector times the level factor 1 << fsh
__device__ __forceinline__ int2 ssd_centre(const int2 *__restrict__ parent, int pty, int ptx, int fsh, int tx, int ty,
                                           int T, int f) {
    if (!parent) return make_int2(0, 0);
    const int px = min(((tx * T + T / 2) >> fsh) / T, ptx - 1);
    const int py = min(((ty * T + T / 2) >> fsh) / T, pty - 1);
    const int2 pv = HMFSR_LDG(parent + (size_t)f * pty * ptx + (size_t)py * ptx + px);
    return make_int2(pv.x << fsh, pv.y << fsh);
}

// N consecutive values of one level row from column x.  inside: every column lies in the
// row, so the reads index one base pointer.  Otherwise each column is clamped to the row;
// an opaque copy of x makes the clamps be recomputed at each call instead of all N clamped
// offsets being held in registers across the caller's loop.
template <int N>
__device__ __forceinline__ void load_row(const uint16_t *__restrict__ row, int x, int lw, bool inside, int (&v)[N]) {
    if (inside) {
#pragma unroll
        for (int i = 0; i < N; ++i) v[i] = HMFSR_LDG(row + x + i);
    } else {
        int xb = x;
        asm volatile("" : "+r"(xb));
#pragma unroll
        for (int i = 0; i < N; ++i) v[i] = HMFSR_LDG(row + clampi(xb + i, 0, lw - 1));
    }
}

// N consecutive values of one level row from column x through whole 16-byte loads: the
// chunks that cover [x, x + N) are read and the N values picked out at the run-time offset
// x mod 8 (selects on its bits, then a 16-bit funnel shift), so a warp's loads touch each
// sector once instead of once per 2-byte value.  Needs a row that starts on a 16-byte
// boundary and 0 <= x, x + N <= its width (a multiple of 8), so no chunk leaves the row.
// kX8: x is a multiple of 8 (no picking).
template <int N, bool kX8 = false>
__device__ __forceinline__ void load_row_vec(const uint16_t *__restrict__ row, int x, int (&v)[N]) {
    if constexpr (kX8) {
        static_assert(N % 8 == 0, "whole chunks");
        const uint4 *p = reinterpret_cast<const uint4 *>(row + x);
#pragma unroll
        for (int c = 0; c < N / 8; ++c) {
            const uint4 q = HMFSR_LDG(p + c);
            const uint32_t w[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                v[8 * c + 2 * k] = (int)(w[k] & 0xffffu);
                v[8 * c + 2 * k + 1] = (int)(w[k] >> 16);
            }
        }
    } else {
        constexpr int kC = (N + 14) / 8;  // chunks at the largest offset, 7
        constexpr int kO = (N + 1) / 2;   // 32-bit words of output
        static_assert(kO + 3 < 4 * kC, "the selects stay inside the loaded words");
        const int s = x & 7;
        const uint4 *p = reinterpret_cast<const uint4 *>(row + (x - s));
        uint32_t w[4 * kC];
#pragma unroll
        for (int c = 0; c < kC; ++c) {
            // chunk c holds values 8 c - s .. 8 c - s + 7 of the span: needed iff 8 c < s + N
            uint4 q = make_uint4(0u, 0u, 0u, 0u);
            if (c < kC - 1 || s + N > 8 * c) q = HMFSR_LDG(p + c);
            w[4 * c] = q.x;
            w[4 * c + 1] = q.y;
            w[4 * c + 2] = q.z;
            w[4 * c + 3] = q.w;
        }
        const int qw = s >> 1;
        const unsigned int sh = (unsigned int)(s & 1) * 16u;
        uint32_t X[kO + 1];  // X[m] = w[qw + m]
#pragma unroll
        for (int m = 0; m <= kO; ++m) {
            const uint32_t a = (qw & 1) ? w[m + 1] : w[m];
            const uint32_t b = (qw & 1) ? w[m + 3] : w[m + 2];
            X[m] = (qw & 2) ? b : a;
        }
#pragma unroll
        for (int k = 0; k < kO; ++k) {
            const uint32_t W = __funnelshift_r(X[k], X[k + 1], sh);
            v[2 * k] = (int)(W & 0xffffu);
            if (2 * k + 1 < N) v[2 * k + 1] = (int)(W >> 16);
        }
    }
}

// load_row, through load_row_vec where `vec` says the rows are 16-byte aligned and the span
// lies inside the row
template <int N, bool kX8 = false>
__device__ __forceinline__ void load_row2(const uint16_t *__restrict__ row, int x, int lw, bool inside, bool vec,
                                          int (&v)[N]) {
    if (vec) load_row_vec<N, kX8>(row, x, v);
    else load_row(row, x, lw, inside, v);
}

// a level's rows start on 16-byte boundaries
__device__ __forceinline__ bool rows_aligned16(const uint16_t *img, int lw) {
    return (lw & 7) == 0 && (reinterpret_cast<uintptr_t>(img) & 15) == 0;
}

// the tile's columns x0 .. x0 + T - 1 and its candidates' xa .. xa + T + 2 RAD - 1 all lie
// inside a level row of lw texels
__device__ __forceinline__ bool ssd_inside(int x0, int xa, int T, int RAD, int lw) {
    return xa >= 0 && xa + T + 2 * RAD <= lw && x0 + T <= lw;
}

// One thread per tile of one level: exhaustive integer SSD over offsets |d| <= RAD
// around the candidate (the parent's vector times the level factor).  For each dy the
// thread streams the tile's rows (L1-cached reads, clamped at the border) and keeps the
// 2 RAD + 1 candidate sums of that row of offsets in registers.  Ties: smallest SSD,
// then smallest |dx| + |dy|, then smaller dy, then smaller dx -- one 64-bit key whose
// minimum decides.
template <int T, int RAD, int PART = 4>
__device__ __forceinline__ void ssd(const uint16_t *__restrict__ img, int lh, int lw, int lty, int ltx,
                                    const int2 *__restrict__ parent, int pty, int ptx, int fsh, int ref,
                                    int2 *__restrict__ vec, int tile, int f) {
    constexpr int kW = 2 * RAD + 1;
    if (tile >= lty * ltx) return;
    const int ty = tile / ltx, tx = tile - ty * ltx;
    int2 *out = vec + (size_t)f * lty * ltx + tile;
    if (f == ref) {
        HMFSR_ST(out, make_int2(0, 0));
        return;
    }
    const int2 cc = ssd_centre(parent, pty, ptx, fsh, tx, ty, T, f);
    const int cx = cc.x, cy = cc.y;
    const uint16_t *R = img + (size_t)ref * lh * lw;
    const uint16_t *A = img + (size_t)f * lh * lw;
    const int x0 = tx * T, y0 = ty * T, xa = x0 + cx - RAD;
    const bool inside = ssd_inside(x0, xa, T, RAD, lw);
    const bool vrow = inside && rows_aligned16(img, lw);
    unsigned long long best = ~0ull;
    for (int dy = -RAD; dy <= RAD; ++dy) {
        SsdAcc<T, PART> acc[kW];
        for (int j = 0; j < T; ++j) {
            const uint16_t *rrow = R + (size_t)min(y0 + j, lh - 1) * lw;
            const uint16_t *arow = A + (size_t)clampi(y0 + j + cy + dy, 0, lh - 1) * lw;
            int rv[T], av[T + 2 * RAD];
            load_row2<T, T % 8 == 0>(rrow, x0, lw, inside, vrow, rv);
            load_row2(arow, xa, lw, inside, vrow, av);
#pragma unroll
            for (int k = 0; k < kW; ++k) acc[k].add(rv, av + k, j);
        }
#pragma unroll
        for (int k = 0; k < kW; ++k) {
            const unsigned long long key = ssd_key(acc[k].total, k - RAD, dy);
            best = key < best ? key : best;
        }
    }
    const int bdx = (int)(best & 15ull) - 7, bdy = (int)((best >> 4) & 15ull) - 7;
    HMFSR_ST(out, make_int2(cx + bdx, cy + bdy));
}

// The same search with the tile rows outermost (small radii): each candidate row is read
// once and serves the 2 RAD + 1 offsets dy that use it; a rolling window of 2 RAD + 1
// candidate rows stays in registers.  Same sums and keys as ssd(), so the same vector.
template <int T, int RAD, int PART = 4>
__device__ __forceinline__ void ssd_rows(const uint16_t *__restrict__ img, int lh, int lw, int lty, int ltx,
                                         const int2 *__restrict__ parent, int pty, int ptx, int fsh, int ref,
                                         int2 *__restrict__ vec, int tile, int f) {
    constexpr int kW = 2 * RAD + 1, kA = T + 2 * RAD;
    if (tile >= lty * ltx) return;
    const int ty = tile / ltx, tx = tile - ty * ltx;
    int2 *out = vec + (size_t)f * lty * ltx + tile;
    if (f == ref) {
        HMFSR_ST(out, make_int2(0, 0));
        return;
    }
    const int2 cc = ssd_centre(parent, pty, ptx, fsh, tx, ty, T, f);
    const uint16_t *R = img + (size_t)ref * lh * lw;
    const uint16_t *A = img + (size_t)f * lh * lw;
    const int x0 = tx * T, y0 = ty * T, xa = x0 + cc.x - RAD;
    const bool inside = ssd_inside(x0, xa, T, RAD, lw);
    // per-thread 16-byte row loads measured slower here (fewer loads in flight); the
    // 2-byte loads of 32 neighbouring tiles share their sectors in L1
    const bool vrow = false;
    SsdAcc<T, PART> acc[kW][kW];
    int av[kW][kA];  // av[d]: candidate row y0 + j + d - RAD (+ the centre's dy)
#pragma unroll
    for (int d = 0; d < kW - 1; ++d) {
        const uint16_t *arow = A + (size_t)clampi(y0 + d - RAD + cc.y, 0, lh - 1) * lw;
        load_row2(arow, xa, lw, inside, vrow, av[d]);
    }
#pragma unroll
    for (int j = 0; j < T; ++j) {
        load_row2(A + (size_t)clampi(y0 + j + RAD + cc.y, 0, lh - 1) * lw, xa, lw, inside, vrow, av[kW - 1]);
        int rv[T];
        load_row2<T, T % 8 == 0>(R + (size_t)min(y0 + j, lh - 1) * lw, x0, lw, inside, vrow, rv);
#pragma unroll
        for (int d = 0; d < kW; ++d)
#pragma unroll
            for (int k = 0; k < kW; ++k) acc[d][k].add(rv, av[d] + k, j);
#pragma unroll
        for (int d = 0; d < kW - 1; ++d)
#pragma unroll
            for (int i = 0; i < kA; ++i) av[d][i] = av[d + 1][i];
    }
    unsigned long long best = ~0ull;
#pragma unroll
    for (int d = 0; d < kW; ++d)
#pragma unroll
        for (int k = 0; k < kW; ++k) {
            const unsigned long long key = ssd_key(acc[d][k].total, k - RAD, d - RAD);
            best = key < best ? key : best;
        }
    const int bdx = (int)(best & 15ull) - 7, bdy = (int)((best >> 4) & 15ull) - 7;
    HMFSR_ST(out, make_int2(cc.x + bdx, cc.y + bdy));
}

// The same search with the offsets dy spread over a group of 2 RAD + 1 lanes (lane d of
// the group takes dy = d - RAD): a warp holds 32 / (2 RAD + 1) groups, one tile each, and
// its remaining lanes idle.  Each lane gathers the group's keys by shuffles and takes
// their minimum; the group's first lane writes.  Every lane of the warp calls this; f is
// the same for the whole warp.
template <int T, int RAD, int PART = 4>
__device__ __forceinline__ void ssd_group(const uint16_t *__restrict__ img, int lh, int lw, int lty, int ltx,
                                          const int2 *__restrict__ parent, int pty, int ptx, int fsh, int ref,
                                          int2 *__restrict__ vec, int tile0, int lane, int f) {
    constexpr int kW = 2 * RAD + 1, kG = 32 / kW;
    static_assert(kW <= 16, "at least two groups per warp");
    const int grp = lane / kW, d = lane - grp * kW;
    const int tile = tile0 + grp;
    const bool active = grp < kG && tile < lty * ltx;
    if (f == ref) {
        if (active && d == 0) HMFSR_ST(vec + (size_t)f * lty * ltx + tile, make_int2(0, 0));
        return;
    }
    const int ty = active ? tile / ltx : 0, tx = active ? tile - (tile / ltx) * ltx : 0;
    const int2 cc = active ? ssd_centre(parent, pty, ptx, fsh, tx, ty, T, f) : make_int2(0, 0);
    unsigned long long best = ~0ull;
    if (active) {
        const int dy = d - RAD;
        const uint16_t *R = img + (size_t)ref * lh * lw;
        const uint16_t *A = img + (size_t)f * lh * lw;
        const int x0 = tx * T, y0 = ty * T, xa = x0 + cc.x - RAD;
        const bool inside = ssd_inside(x0, xa, T, RAD, lw);
        const bool vrow = inside && rows_aligned16(img, lw);
        SsdAcc<T, PART> acc[kW];
        for (int j = 0; j < T; ++j) {
            const uint16_t *rrow = R + (size_t)min(y0 + j, lh - 1) * lw;
            const uint16_t *arow = A + (size_t)clampi(y0 + j + cc.y + dy, 0, lh - 1) * lw;
            int rv[T], av[T + 2 * RAD];
            load_row2<T, T % 8 == 0>(rrow, x0, lw, inside, vrow, rv);
            load_row2(arow, xa, lw, inside, vrow, av);
#pragma unroll
            for (int k = 0; k < kW; ++k) acc[k].add(rv, av + k, j);
        }
#pragma unroll
        for (int k = 0; k < kW; ++k) {
            const unsigned long long key = ssd_key(acc[k].total, k - RAD, dy);
            best = key < best ? key : best;
        }
    }
    // idle lanes read the last group (their result is unused)
    const int base = min(grp, kG - 1) * kW;
    unsigned long long m = ~0ull;
#pragma unroll
    for (int k = 0; k < kW; ++k) {
        const unsigned long long o = __shfl_sync(0xffffffffu, best, base + k);
        m = o < m ? o : m;
    }
    if (active && d == 0) {
        const int bdx = (int)(m & 15ull) - 7, bdy = (int)((m >> 4) & 15ull) - 7;
        HMFSR_ST(vec + (size_t)f * lty * ltx + tile, make_int2(cc.x + bdx, cc.y + bdy));
    }
}

// Lucas-Kanade refinement (Sec. 3.2) of one level-0 tile per warp, on I = Lq / 4.  Each
// lane owns pixels lane + 32 m of the tile.  Gradients of the base frame by central
// differences around the clamped pixel; H = sum g g^T is summed exactly in integers, so
// the conditioning guard (tr H == 0 or det H <= 1e-9 tr(H)^2) is an exact 128-bit integer
// test; each iteration accumulates sum g r in FP32 (warp shuffles) and solves the 2x2
// system.
template <int T>
__device__ __forceinline__ void lk(const uint16_t *__restrict__ L0, int lh, int lw, int lty, int ltx,
                                   const int2 *__restrict__ vec0, int ref, int iters, float *__restrict__ motion,
                                   int32_t *__restrict__ motion_int, int warp, int lane, int f) {
    constexpr int t = T, npx = T * T, nper = (npx + 31) / 32;
    if (warp >= lty * ltx) return;
    const int ty = warp / ltx, tx = warp % ltx;
    const size_t o = (size_t)f * lty * ltx + warp;
    if (f == ref) {
        if (lane == 0) {
            HMFSR_ST(motion + 2 * o, 0.f);
            HMFSR_ST(motion + 2 * o + 1, 0.f);
            if (motion_int) { HMFSR_ST(motion_int + 2 * o, 0); HMFSR_ST(motion_int + 2 * o + 1, 0); }
        }
        return;
    }
    const uint16_t *R = L0 + (size_t)ref * lh * lw;
    const uint16_t *A = L0 + (size_t)f * lh * lw;
    const int2 u = HMFSR_LD(vec0 + o);
    int gxs[nper], gys[nper], pxs[nper], pys[nper], rv[nper];
    long long hxx = 0, hxy = 0, hyy = 0;
#pragma unroll
    for (int m = 0; m < nper; ++m) {
        const int k = lane + 32 * m;
        if (k >= npx) { gxs[m] = gys[m] = 0; pxs[m] = pys[m] = 0; rv[m] = 0; continue; }
        const int x = min(tx * t + k % t, lw - 1), y = min(ty * t + k / t, lh - 1);
        const uint16_t *row = R + (size_t)y * lw;
        const int gx = (int)HMFSR_LDG(row + min(x + 1, lw - 1)) - (int)HMFSR_LDG(row + max(x - 1, 0));
        const int gy = (int)HMFSR_LDG(R + (size_t)min(y + 1, lh - 1) * lw + x) - (int)HMFSR_LDG(R + (size_t)max(y - 1, 0) * lw + x);
        gxs[m] = gx; gys[m] = gy; pxs[m] = x; pys[m] = y;
        rv[m] = HMFSR_LDG(row + x);
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
                const float i00 = HMFSR_LDG(a0 + x0), i10 = HMFSR_LDG(a0 + x1), i01 = HMFSR_LDG(a1 + x0), i11 = HMFSR_LDG(a1 + x1);
                const float top = fmaf(ax, i10, (1.f - ax) * i00), bot = fmaf(ax, i11, (1.f - ax) * i01);
                const float ia = fmaf(ay, bot, (1.f - ay) * top);
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
        HMFSR_ST(motion + 2 * o, 2.f * ((float)u.x + dx));
        HMFSR_ST(motion + 2 * o + 1, 2.f * ((float)u.y + dy));
        if (motion_int) { HMFSR_ST(motion_int + 2 * o, (int32_t)u.x); HMFSR_ST(motion_int + 2 * o + 1, (int32_t)u.y); }
    }
}

// The same refinement with T / 2 lanes per tile (T <= 8, 64 / T tiles per warp): lane c of
// a group owns columns 2 c and 2 c + 1 of the tile and walks its T rows, so neighbouring
// columns share their texels (4 loads per row for the two gradients, 3 per row for the two
// bilinear samples) and the per-tile work of the solve is repeated in fewer lanes.  The
// gradient rows roll down the tile where no row is clamped (the tile ends inside the
// level).  Sums over the group by butterfly shuffles inside the group; every lane of the
// warp runs every iteration (a skipped or absent tile adds nothing and keeps its vector),
// so the shuffles stay converged.  f is the same for the whole warp.
// Level-0 block matching at radius 1 by a tile's T / 2 refinement lanes (f != ref): lane c
// of the group sums the squared differences of the tile's columns 2 c and 2 c + 1 for the
// 9 offsets, rolling over the T + 2 candidate rows it reads (4 columns each); butterfly
// sums inside the group give every lane the tile's 9 exact sums, and the first-minimum
// key picks the vector.  The sums, the keys and the clamping are those of ssd_rows, so the
// vector is the same.  Every lane of the warp calls this.
template <int T, int PART>
__device__ __forceinline__ int2 ssd0_lanes(const uint16_t *__restrict__ img, int lh, int lw, int lty, int ltx,
                                           const int2 *__restrict__ parent, int pty, int ptx, int fsh, int ref,
                                           int tile, int lane, int f) {
    static_assert(T == 4 || T == 8, "T / 2 lanes per tile");
    constexpr int kL = T / 2;
    constexpr int kRows = PART >= 2 * T ? T : PART / 2;  // rows per 32-bit partial (2 terms a row)
    const int c = 2 * (lane & (kL - 1));
    const bool active = tile < lty * ltx;
    const int ty = active ? tile / ltx : 0, tx = active ? tile - (tile / ltx) * ltx : 0;
    const int2 cc = active ? ssd_centre(parent, pty, ptx, fsh, tx, ty, T, f) : make_int2(0, 0);
    const uint16_t *R = img + (size_t)ref * lh * lw;
    const uint16_t *A = img + (size_t)f * lh * lw;
    const int x0 = tx * T, y0 = ty * T;
    const int rc0 = min(x0 + c, lw - 1), rc1 = min(x0 + c + 1, lw - 1);
    int ac[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) ac[k] = clampi(x0 + cc.x - 1 + c + k, 0, lw - 1);
    const int ya = y0 + cc.y - 1;  // candidate row r of the window is ya + r, r = 0 .. T + 1
    int av[3][4];
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        const uint16_t *row = A + clampi(ya + r, 0, lh - 1) * lw;
#pragma unroll
        for (int k = 0; k < 4; ++k) av[r][k] = HMFSR_LDG(row + ac[k]);
    }
    unsigned long long tot[3][3];
    unsigned int part[3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) { tot[a][b] = 0ull; part[a][b] = 0u; }
#pragma unroll
    for (int j = 0; j < T; ++j) {
        const uint16_t *row = A + clampi(ya + j + 2, 0, lh - 1) * lw;
#pragma unroll
        for (int k = 0; k < 4; ++k) av[2][k] = HMFSR_LDG(row + ac[k]);
        const uint16_t *rrow = R + min(y0 + j, lh - 1) * lw;
        const int rv0 = HMFSR_LDG(rrow + rc0), rv1 = HMFSR_LDG(rrow + rc1);
#pragma unroll
        for (int dyi = 0; dyi < 3; ++dyi)
#pragma unroll
            for (int dxi = 0; dxi < 3; ++dxi) {
                const int d0 = rv0 - av[dyi][dxi], d1 = rv1 - av[dyi][dxi + 1];
                part[dyi][dxi] += (unsigned int)(d0 * d0) + (unsigned int)(d1 * d1);
            }
        if ((j + 1) % kRows == 0 || j == T - 1) {
#pragma unroll
            for (int a = 0; a < 3; ++a)
#pragma unroll
                for (int b = 0; b < 3; ++b) { tot[a][b] += part[a][b]; part[a][b] = 0u; }
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) { av[0][k] = av[1][k]; av[1][k] = av[2][k]; }
    }
    unsigned long long best = ~0ull;
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            unsigned long long v = tot[a][b];
#pragma unroll
            for (int m = kL / 2; m > 0; m >>= 1) v += __shfl_xor_sync(0xffffffffu, v, m);
            const unsigned long long key = ssd_key(v, b - 1, a - 1);
            best = key < best ? key : best;
        }
    const int bdx = (int)(best & 15ull) - 7, bdy = (int)((best >> 4) & 15ull) - 7;
    return make_int2(cc.x + bdx, cc.y + bdy);
}

// the refinement of one tile from its integer vector u (f != ref); lk_group below reads u
// from the level-0 vectors, the fused search-and-refine kernel passes the one it found
template <int T>
__device__ __forceinline__ void lk_group_u(const uint16_t *__restrict__ L0, int lh, int lw, int lty, int ltx, int ref,
                                           int iters, float *__restrict__ motion, int32_t *__restrict__ motion_int,
                                           int tile, int lane, int f, int2 u) {
    static_assert(T == 4 || T == 8, "T / 2 lanes per tile");
    constexpr int kL = T / 2;
    const int c = 2 * (lane & (kL - 1));
    const bool active = tile < lty * ltx;
    const size_t o = (size_t)f * lty * ltx + tile;
    const int ty = active ? tile / ltx : 0, tx = active ? tile - (tile / ltx) * ltx : 0;
    const uint16_t *R = L0 + (size_t)ref * lh * lw;
    const uint16_t *A = L0 + (size_t)f * lh * lw;
    // the lane's two pixel columns (clamped into the level) and their gradient neighbours:
    // x0 + 1 is x1's column or, where both clamp to the last column, x0 itself
    const int x0 = min(tx * T + c, lw - 1), x1 = min(tx * T + c + 1, lw - 1);
    const int xm = max(x0 - 1, 0), xp = min(x1 + 1, lw - 1);
    const bool same = (x1 == x0);
    const int y0 = ty * T;
    float gxs[2 * T], gys[2 * T], rv[2 * T];
    long long hxx = 0, hxy = 0, hyy = 0;
    {
        const bool roll = (y0 + T <= lh);
        int pm0 = 0, pm1 = 0, c0 = 0, c1 = 0;
        if (roll) {
            const uint16_t *rm = R + max(y0 - 1, 0) * lw, *rc = R + y0 * lw;
            pm0 = HMFSR_LDG(rm + x0); pm1 = HMFSR_LDG(rm + x1);
            c0 = HMFSR_LDG(rc + x0); c1 = HMFSR_LDG(rc + x1);
        }
#pragma unroll
        for (int j = 0; j < T; ++j) {
            const int y = min(y0 + j, lh - 1);
            const uint16_t *row = R + y * lw;  // 32-bit offsets: a level holds < 2^31 texels
            if (!roll) {
                const uint16_t *rm = R + max(y - 1, 0) * lw;
                pm0 = HMFSR_LDG(rm + x0); pm1 = HMFSR_LDG(rm + x1);
                c0 = HMFSR_LDG(row + x0); c1 = HMFSR_LDG(row + x1);
            }
            const uint16_t *rp = R + min(y + 1, lh - 1) * lw;
            const int n0 = HMFSR_LDG(rp + x0), n1 = HMFSR_LDG(rp + x1);
            const int lm = HMFSR_LDG(row + xm), lp = HMFSR_LDG(row + xp);
            const int gx0 = c1 - lm, gx1 = lp - (same ? lm : c0);
            const int gy0 = n0 - pm0, gy1 = n1 - pm1;
            gxs[2 * j] = (float)gx0 * 0.125f;
            gxs[2 * j + 1] = (float)gx1 * 0.125f;
            gys[2 * j] = (float)gy0 * 0.125f;
            gys[2 * j + 1] = (float)gy1 * 0.125f;
            rv[2 * j] = (float)c0;
            rv[2 * j + 1] = (float)c1;
            // |g| < 2^15: two squares or products fit a 32-bit int
            hxx += (long long)(gx0 * gx0 + gx1 * gx1);
            hxy += (long long)(gx0 * gy0 + gx1 * gy1);
            hyy += (long long)(gy0 * gy0 + gy1 * gy1);
            pm0 = c0; pm1 = c1;
            c0 = n0; c1 = n1;
        }
    }
#pragma unroll
    for (int m = kL / 2; m > 0; m >>= 1) {
        hxx += __shfl_xor_sync(0xffffffffu, hxx, m);
        hxy += __shfl_xor_sync(0xffffffffu, hxy, m);
        hyy += __shfl_xor_sync(0xffffffffu, hyy, m);
    }
    // conditioning guard, exact: skip when tr H == 0 or 10^9 det H <= tr(H)^2
    const __int128 det_i = (__int128)hxx * hyy - (__int128)hxy * hxy;
    const __int128 tr_i = (__int128)hxx + hyy;
    const bool skip = (tr_i == 0) || ((__int128)1000000000 * det_i <= tr_i * tr_i);
    // H in units of g = (Lq difference) / 8 is H_int / 64
    const float Hxx = (float)hxx, Hxy = (float)hxy, Hyy = (float)hyy;
    const float inv = skip ? 0.f : 64.f / fmaf(Hxx, Hyy, -Hxy * Hxy);
    float dx = 0.f, dy = 0.f;
    for (int it = 0; it < iters; ++it) {
        const float fdx = floorf(dx), fdy = floorf(dy);
        const float ax = dx - fdx, ay = dy - fdy;
        const int ox = u.x + (int)fdx, oy = u.y + (int)fdy;
        // sample columns: pixel 0 between s0 and s1, pixel 1 between s1 and s2 (or, where
        // both pixels are the clamped last column, between s0 and s1 as well)
        const int s0 = clampi(x0 + ox, 0, lw - 1), s1 = clampi(x0 + ox + 1, 0, lw - 1);
        const int s2 = clampi(x1 + ox + 1, 0, lw - 1);
        float bx = 0.f, by = 0.f;
        if (y0 + T <= lh && y0 + oy >= 0 && y0 + oy + T < lh) {
            // the tile's rows and the sampled rows are inside the level: one row after another
            const uint16_t *a = A + (y0 + oy) * lw;
            float t0 = (float)HMFSR_LDG(a + s0), t1 = (float)HMFSR_LDG(a + s1), t2 = (float)HMFSR_LDG(a + s2);
#pragma unroll
            for (int j = 0; j < T; ++j) {
                a += lw;
                const float b0 = (float)HMFSR_LDG(a + s0), b1 = (float)HMFSR_LDG(a + s1), b2 = (float)HMFSR_LDG(a + s2);
                const float top0 = fmaf(ax, t1, (1.f - ax) * t0), bot0 = fmaf(ax, b1, (1.f - ax) * b0);
                const float top1 = same ? top0 : fmaf(ax, t2, (1.f - ax) * t1);
                const float bot1 = same ? bot0 : fmaf(ax, b2, (1.f - ax) * b1);
                const float ia0 = fmaf(ay, bot0, (1.f - ay) * top0), ia1 = fmaf(ay, bot1, (1.f - ay) * top1);
                const float r0 = (ia0 - rv[2 * j]) * 0.25f, r1 = (ia1 - rv[2 * j + 1]) * 0.25f;
                bx = fmaf(gxs[2 * j], r0, bx);
                by = fmaf(gys[2 * j], r0, by);
                bx = fmaf(gxs[2 * j + 1], r1, bx);
                by = fmaf(gys[2 * j + 1], r1, by);
                t0 = b0; t1 = b1; t2 = b2;
            }
        } else {
#pragma unroll
            for (int j = 0; j < T; ++j) {
                const int iy = min(y0 + j, lh - 1) + oy;
                const uint16_t *a0 = A + clampi(iy, 0, lh - 1) * lw;
                const uint16_t *a1 = A + clampi(iy + 1, 0, lh - 1) * lw;
                const float t0 = (float)HMFSR_LDG(a0 + s0), t1 = (float)HMFSR_LDG(a0 + s1), t2 = (float)HMFSR_LDG(a0 + s2);
                const float b0 = (float)HMFSR_LDG(a1 + s0), b1 = (float)HMFSR_LDG(a1 + s1), b2 = (float)HMFSR_LDG(a1 + s2);
                const float top0 = fmaf(ax, t1, (1.f - ax) * t0), bot0 = fmaf(ax, b1, (1.f - ax) * b0);
                const float top1 = same ? top0 : fmaf(ax, t2, (1.f - ax) * t1);
                const float bot1 = same ? bot0 : fmaf(ax, b2, (1.f - ax) * b1);
                const float ia0 = fmaf(ay, bot0, (1.f - ay) * top0), ia1 = fmaf(ay, bot1, (1.f - ay) * top1);
                const float r0 = (ia0 - rv[2 * j]) * 0.25f, r1 = (ia1 - rv[2 * j + 1]) * 0.25f;
                bx = fmaf(gxs[2 * j], r0, bx);
                by = fmaf(gys[2 * j], r0, by);
                bx = fmaf(gxs[2 * j + 1], r1, bx);
                by = fmaf(gys[2 * j + 1], r1, by);
            }
        }
#pragma unroll
        for (int m = kL / 2; m > 0; m >>= 1) {
            bx += __shfl_xor_sync(0xffffffffu, bx, m);
            by += __shfl_xor_sync(0xffffffffu, by, m);
        }
        if (!skip) {
            const float sx = -(Hyy * bx - Hxy * by) * inv;
            const float sy = -(Hxx * by - Hxy * bx) * inv;
            dx = fminf(fmaxf(dx + sx, -1.f), 1.f);
            dy = fminf(fmaxf(dy + sy, -1.f), 1.f);
        }
    }
    if (active && c == 0) {
        HMFSR_ST(motion + 2 * o, 2.f * ((float)u.x + dx));
        HMFSR_ST(motion + 2 * o + 1, 2.f * ((float)u.y + dy));
        if (motion_int) { HMFSR_ST(motion_int + 2 * o, (int32_t)u.x); HMFSR_ST(motion_int + 2 * o + 1, (int32_t)u.y); }
    }
}

template <int T>
__device__ __forceinline__ void lk_group(const uint16_t *__restrict__ L0, int lh, int lw, int lty, int ltx,
                                         const int2 *__restrict__ vec0, int ref, int iters, float *__restrict__ motion,
                                         int32_t *__restrict__ motion_int, int tile, int lane, int f) {
    constexpr int kL = T / 2;
    const int c = 2 * (lane & (kL - 1));
    const bool active = tile < lty * ltx;
    const size_t o = (size_t)f * lty * ltx + tile;
    if (f == ref) {
        if (active && c == 0) {
            HMFSR_ST(motion + 2 * o, 0.f);
            HMFSR_ST(motion + 2 * o + 1, 0.f);
            if (motion_int) { HMFSR_ST(motion_int + 2 * o, 0); HMFSR_ST(motion_int + 2 * o + 1, 0); }
        }
        return;
    }
    const int2 u = active ? HMFSR_LD(vec0 + o) : make_int2(0, 0);
    lk_group_u<T>(L0, lh, lw, lty, ltx, ref, iters, motion, motion_int, tile, lane, f, u);
}

// Subpixel refinement by a quadratic fit (Sec. 3.2: the variant the paper explored before
// Lucas-Kanade), one thread per level-0 tile: the exact SSD at the integer vector and at
// its neighbours along each axis, and per axis the vertex of the parabola through the
// three, (E- - E+) / (2 (E- - 2 E0 + E+)), 0 unless the curvature is positive, clamped to
// [-1/2, 1/2].  FP64 from exact integers, so the result is the same bits as an FP64
// restatement on the CPU.
__device__ __forceinline__ double parabola_vertex(long long em, long long e0, long long ep) {
    const long long den = 2 * (em - 2 * e0 + ep);
    if (den <= 0) return 0.0;
    return fmin(fmax(__ddiv_rn((double)(em - ep), (double)den), -0.5), 0.5);
}

template <int T>
__device__ __forceinline__ void quadfit(const uint16_t *__restrict__ L0, int lh, int lw, int lty, int ltx,
                                        const int2 *__restrict__ vec0, int ref, float *__restrict__ motion,
                                        int32_t *__restrict__ motion_int, int tile, int f) {
    if (tile >= lty * ltx) return;
    const size_t o = (size_t)f * lty * ltx + tile;
    if (f == ref) {
        HMFSR_ST(motion + 2 * o, 0.f);
        HMFSR_ST(motion + 2 * o + 1, 0.f);
        if (motion_int) { HMFSR_ST(motion_int + 2 * o, 0); HMFSR_ST(motion_int + 2 * o + 1, 0); }
        return;
    }
    const int ty = tile / ltx, tx = tile - ty * ltx;
    const uint16_t *R = L0 + (size_t)ref * lh * lw;
    const uint16_t *A = L0 + (size_t)f * lh * lw;
    const int2 u = HMFSR_LD(vec0 + o);
    const int x0 = tx * T, y0 = ty * T;
    auto ssd_at = [&](int dx, int dy) -> long long {
        long long e = 0;
        for (int j = 0; j < T; ++j) {
            const uint16_t *rr = R + min(y0 + j, lh - 1) * lw;
            const uint16_t *ar = A + clampi(y0 + j + u.y + dy, 0, lh - 1) * lw;
#pragma unroll
            for (int i = 0; i < T; ++i) {
                const int d = (int)HMFSR_LDG(rr + min(x0 + i, lw - 1)) - (int)HMFSR_LDG(ar + clampi(x0 + i + u.x + dx, 0, lw - 1));
                e += (long long)(d * d);
            }
        }
        return e;
    };
    const long long e0 = ssd_at(0, 0);
    const double dx = parabola_vertex(ssd_at(-1, 0), e0, ssd_at(1, 0));
    const double dy = parabola_vertex(ssd_at(0, -1), e0, ssd_at(0, 1));
    HMFSR_ST(motion + 2 * o, (float)__dmul_rn(2.0, __dadd_rn((double)u.x, dx)));
    HMFSR_ST(motion + 2 * o + 1, (float)__dmul_rn(2.0, __dadd_rn((double)u.y, dy)));
    if (motion_int) { HMFSR_ST(motion_int + 2 * o, (int32_t)u.x); HMFSR_ST(motion_int + 2 * o + 1, (int32_t)u.y); }
}

// ======================================================================================
// merge preparation (Sec. 5.1.2, 5.2)
// ======================================================================================
// --------------------------------------------------------------------------------------
// noise-corrected statistics of the base frame that do not depend on the other frame
// (Eq. 6, closed-form noise model), from the 3x3 guide sums S1 and sums of squares S2
// --------------------------------------------------------------------------------------
__device__ __forceinline__ float4 base_stats_of(const uint32_t (&S1)[3], const uint32_t (&S2)[3], const MergeConsts &c,
                                                int wl) {
    float sig2 = 0.f, dmd2[3];
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) {
        // green guide = (G1 + G2) / 2
        long long num = 9LL * (long long)S2[ch] - (long long)S1[ch] * (long long)S1[ch];
        const float igs = (ch == 1) ? 0.5f : 1.f;
        float var_ms = fmaxf((float)num * (igs * igs * (1.f / 81.f)), 0.f);
        float mu = (float)S1[ch] * (igs * (1.f / 9.f));
        float var_md;
        if (c.noise_table) {
            // Monte-Carlo statistics, linear between the brightness levels around mu
            const float tp = fminf(fmaxf(mu, 0.f), (float)wl) * ((float)(kNoiseLevels - 1) / (float)wl);
            const int i = min((int)tp, kNoiseLevels - 2);
            const float f = tp - (float)i;
            const float4 t0 = HMFSR_LDG(c.noise_table + i), t1 = HMFSR_LDG(c.noise_table + i + 1);
            const float v0 = ch == 1 ? t0.y : t0.x, v1 = ch == 1 ? t1.y : t1.x;
            const float d0 = ch == 1 ? t0.w : t0.z, d1 = ch == 1 ? t1.w : t1.z;
            var_md = fmaf(f, v1 - v0, v0);
            dmd2[ch] = fmaf(f, d1 - d0, d0);
        } else {
            var_md = fmaxf(fmaf(c.noise_a, fminf(fmaxf(mu, 0.f), (float)wl), c.noise_b) * igs, 0.f);
            dmd2[ch] = var_md * (2.f / 9.f);
        }
        sig2 += fmaxf(var_ms, var_md);
    }
    float eps = 1e-12f * (float)wl * (float)wl;
    return make_float4(fmaxf(sig2, eps), dmd2[0], dmd2[1], dmd2[2]);
}

// --------------------------------------------------------------------------------------
// structure tensor -> kernel covariance (Eq. 3, Eq. 4, supplement S.1), from the exact
// integer tensor {sum gx^2, sum gx gy, sum gy^2} of the four 2x2 sub-squares
// --------------------------------------------------------------------------------------
// inv_dtr = 1 / (16 WL D_tr)
__device__ __forceinline__ float4 kern_of_tensor(long long ta, long long tb, long long tc, const MergeConsts &c,
                                                 float inv_dtr) {
    // eigen-analysis: lambda1 = (tr + r)/2, dominant direction at angle theta with
    // cos 2theta = (a-c)/r, sin 2theta = 2b/r (theta = 0 when the tensor is isotropic)
    float tr = (float)(ta + tc);
    float amc = (float)(ta - tc), b2 = 2.f * (float)tb;
    float r = fast_sqrt(fmaf(amc, amc, b2 * b2));
    float cs = 1.f, sn = 0.f;
    if (!(ta == tc && tb == 0)) { const float ir = fast_rcp(r); cs = amc * ir; sn = b2 * ir; }
    float l1 = 0.5f * (tr + r);
    float A = (ta + tc == 0) ? 1.f : 1.f + fast_sqrt(r * fast_rcp(tr));
    // lambda in units of luminance normalised to [0,1]: sqrt(l1_norm) = sqrt(l1) / (16 WL)
    float D = fminf(fmaxf(fmaf(-fast_sqrt(l1), inv_dtr, 1.f) + c.d_th, 0.f), 1.f);
    float kh_al = c.k_detail * (c.k_stretch * A);
    float kh_ac = c.k_detail * fast_rcp(c.k_shrink * A);
    float kd = c.k_detail * c.k_denoise;
    float s_al = fmaf(1.f - D, kh_al, D * kd);   // standard deviations before squaring
    float s_ac = fmaf(1.f - D, kh_ac, D * kd);
    float k_al = s_al * s_al, k_ac = s_ac * s_ac;
    // half-angle unit vector e1 = (cos theta, sin theta), without cancellation
    float e1x, e1y;
    {
        // the larger component from sqrt((1 + |cos 2theta|) / 2), the other from sin 2theta / 2x
        // it; -0.5 cs for cs < 0 is the same product as 0.5 |cs|, so these are the same values
        const float big = fast_sqrt(fmaf(0.5f, fabsf(cs), 0.5f));
        const float other = sn * fast_rcp(2.f * big);
        const bool pos = cs >= 0.f;
        e1x = pos ? big : other;
        e1y = pos ? other : big;
    }
    // Omega = k_across e1 e1^T + k_along e2 e2^T (stretch along the edge, e2)
    //       = min I + |k_along - k_across| u u^T with u = e2 if k_along >= k_across else e1
    float dh = (1.f - D) * (kh_al - kh_ac) * (s_al + s_ac);  // k_along - k_across, no cancellation
    if (dh >= 0.f) return make_float4(k_ac, dh, -e1y, e1x);
    return make_float4(k_al, -dh, e1x, e1y);
}

// --------------------------------------------------------------------------------------
// merge preparation of one strip of half-res texels of one frame (Sec. 5.1.2, Sec. 5.2.2,
// Eq. 3-4, supplement S.1): one warp, 32 consecutive texel columns, a strip of rows.
// Each lane builds the guide quad {R, G1+G2, B, Lq} of its column from the raw samples
// row by row (the guide image never goes to memory); the left and right neighbours come
// from the adjacent lanes (lanes 0 and 31 read the strip's halo quads), rows and
// columns clamped at the frame border.  A rolling window over three rows gives the 3x3
// guide sums (and, for the base frame, the noise-corrected statistics of Eq. 6) and the
// exact integer structure tensor of the 3x3 Lq window (forward differences on its four
// 2x2 sub-squares) -> kernel covariance.  Raw rows are fetched two rows ahead.  The R
// and B sums travel packed in one word: 9 x 7281 < 2^16, so the halves never carry.
// --------------------------------------------------------------------------------------
constexpr int kPrepStrip = 32;  // default strip height; per-burst launches choose theirs (strip_rows)

struct PrepRow {
    uint32_t a, b;    // the lane's quad: {R, G1} and {G2, B}
    uint32_t ha, hb;  // lanes 0 and 31: the halo quad beside the strip
};

struct PrepState {
    uint32_t rb[2], gs[2];  // 3-texel row sums of the two previous rows: R | B << 16, G1 + G2
    uint32_t q[2][3];       // 3-texel row sums of squares (base frame)
    int L[3];               // Lq of the previous row at columns -1, 0, +1
    long long pa, pb, pc;   // tensor terms of the previous pair of rows
};

__device__ __forceinline__ PrepRow prep_fetch(const uint16_t *__restrict__ fr, int pitch, int hh, int uc, int uh,
                                              bool halo, int v) {
    const uint16_t *row = fr + (size_t)(2 * clampi(v, 0, hh - 1)) * pitch;
    PrepRow p;
    p.a = HMFSR_LDG(reinterpret_cast<const uint32_t *>(row + 2 * uc));
    p.b = HMFSR_LDG(reinterpret_cast<const uint32_t *>(row + pitch + 2 * uc));
    p.ha = p.hb = 0u;
    if (halo) {
        p.ha = HMFSR_LDG(reinterpret_cast<const uint32_t *>(row + 2 * uh));
        p.hb = HMFSR_LDG(reinterpret_cast<const uint32_t *>(row + pitch + 2 * uh));
    }
    return p;
}

// one raw row pair of the strip (strip row r = -1 .. rows); emits texel row r - 1
__device__ __forceinline__ void prep_row(const PrepRow &p, PrepState &st, int r, int lane, bool is_ref, bool out_col,
                                         int v0, const Geom &g, const MergeConsts &c, float inv_dtr, int u,
                                         uint2 *__restrict__ s1f, float4 *__restrict__ base_stats,
                                         float4 *__restrict__ kernf) {
    const uint32_t R = p.a & 0xffffu, G = (p.a >> 16) + (p.b & 0xffffu), B = p.b >> 16;
    const uint32_t c0 = R | (B << 16), c1 = G | ((R + G + B) << 16);  // {R, B}, {G, Lq}
    uint32_t l0 = __shfl_up_sync(0xffffffffu, c0, 1), l1 = __shfl_up_sync(0xffffffffu, c1, 1);
    uint32_t r0 = __shfl_down_sync(0xffffffffu, c0, 1), r1 = __shfl_down_sync(0xffffffffu, c1, 1);
    {
        // lanes 0 and 31 take the strip's halo quad (p.ha, p.hb; zero in the other lanes)
        const uint32_t hR = p.ha & 0xffffu, hG = (p.ha >> 16) + (p.hb & 0xffffu), hB = p.hb >> 16;
        const uint32_t h0 = hR | (hB << 16), h1 = hG | ((hR + hG + hB) << 16);
        l0 = lane == 0 ? h0 : l0;
        l1 = lane == 0 ? h1 : l1;
        r0 = lane == 31 ? h0 : r0;
        r1 = lane == 31 ? h1 : r1;
    }
    const uint32_t rb = l0 + c0 + r0;                              // R and B halves stay below 2^16
    const uint32_t gs = (l1 & 0xffffu) + G + (r1 & 0xffffu);
    const int L[3] = {(int)(l1 >> 16), (int)(c1 >> 16), (int)(r1 >> 16)};
    uint32_t q[3] = {0u, 0u, 0u};
    if (is_ref) {
        const uint32_t lR = l0 & 0xffffu, lB = l0 >> 16, lG = l1 & 0xffffu;
        const uint32_t rR = r0 & 0xffffu, rB = r0 >> 16, rG = r1 & 0xffffu;
        q[0] = lR * lR + R * R + rR * rR;
        q[1] = lG * lG + G * G + rG * rG;
        q[2] = lB * lB + B * B + rB * rB;
    }
    // tensor terms of the two sub-squares between the previous row and this one
    long long pa = 0, pb = 0, pc = 0;
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const int gx = (st.L[i + 1] - st.L[i]) + (L[i + 1] - L[i]);
        const int gy = (L[i] - st.L[i]) + (L[i + 1] - st.L[i + 1]);
        pa += (long long)gx * gx;
        pb += (long long)gx * gy;
        pc += (long long)gy * gy;
    }
    if (r >= 1 && out_col) {
        const int v = v0 + r - 1;
        if (v < g.hh) {
            const int idx = v * g.wh + u;
            const uint32_t srb = st.rb[0] + st.rb[1] + rb, sg = st.gs[0] + st.gs[1] + gs;
            HMFSR_ST(s1f + idx, make_uint2(srb, sg));
            if (is_ref) {
                const uint32_t S1[3] = {srb & 0xffffu, sg, srb >> 16};
                const uint32_t S2[3] = {st.q[0][0] + st.q[1][0] + q[0], st.q[0][1] + st.q[1][1] + q[1],
                                        st.q[0][2] + st.q[1][2] + q[2]};
                HMFSR_ST(base_stats + idx, base_stats_of(S1, S2, c, g.wl));
            }
            HMFSR_ST(kernf + idx, kern_of_tensor(st.pa + pa, st.pb + pb, st.pc + pc, c, inv_dtr));
        }
    }
    st.rb[0] = st.rb[1]; st.rb[1] = rb;
    st.gs[0] = st.gs[1]; st.gs[1] = gs;
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) { st.q[0][ch] = st.q[1][ch]; st.q[1][ch] = q[ch]; }
#pragma unroll
    for (int i = 0; i < 3; ++i) st.L[i] = L[i];
    st.pa = pa; st.pb = pb; st.pc = pc;
}

// strip (u0 .. u0 + 31) x (v0 .. v0 + rows - 1) of frame f (rows even); every lane of the
// warp calls this (the strip's shuffles need them all)
__device__ __forceinline__ void prep_strip(const uint16_t *__restrict__ burst, const Geom &g, const MergeConsts &c,
                                           uint2 *__restrict__ s1, float4 *__restrict__ base_stats,
                                           float4 *__restrict__ kern, int u0, int v0, int f, int lane,
                                           int rows = kPrepStrip) {
    const uint16_t *fr = burst + (size_t)f * g.h * g.pitch;
    const int u = u0 + lane, uc = min(u, g.wh - 1);
    const bool halo = (lane == 0 || lane == 31);
    const int uh = clampi(lane == 0 ? u0 - 1 : u0 + 32, 0, g.wh - 1);
    const bool is_ref = (f == g.ref), out_col = u < g.wh;
    const size_t hw = (size_t)g.hh * g.wh;
    uint2 *s1f = s1 + (size_t)f * hw;
    float4 *kernf = kern + (size_t)f * hw;
    const float inv_dtr = fast_rcp(16.f * (float)g.wl * c.d_tr);
    PrepState st;
    st.rb[0] = st.rb[1] = st.gs[0] = st.gs[1] = 0u;
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) st.q[0][ch] = st.q[1][ch] = 0u;
    st.L[0] = st.L[1] = st.L[2] = 0;
    st.pa = st.pb = st.pc = 0;
    PrepRow p0 = prep_fetch(fr, g.pitch, g.hh, uc, uh, halo, v0 - 1);
    PrepRow p1 = prep_fetch(fr, g.pitch, g.hh, uc, uh, halo, v0);
    for (int r = -1; r <= rows; r += 2) {
        const PrepRow cur0 = p0;
        p0 = prep_fetch(fr, g.pitch, g.hh, uc, uh, halo, v0 + r + 2);
        prep_row(cur0, st, r, lane, is_ref, out_col, v0, g, c, inv_dtr, u, s1f, base_stats, kernf);
        const PrepRow cur1 = p1;
        p1 = prep_fetch(fr, g.pitch, g.hh, uc, uh, halo, v0 + r + 3);
        prep_row(cur1, st, r + 1, lane, is_ref, out_col, v0, g, c, inv_dtr, u, s1f, base_stats, kernf);
    }
}

// --------------------------------------------------------------------------------------
// motion prior (Eq. 7-8): robustness scale per tile, decided in exact FP64
// --------------------------------------------------------------------------------------
// the motion span M of tile (x, y) and its 3x3 tile neighbourhood exceeds m_th (Eq. 7);
// min / max are exact in FP32; the span, its length and the threshold are FP64
__device__ __forceinline__ bool motion_span_exceeds(const float2 *__restrict__ mv, int ty, int tx, int y, int x,
                                                    float m_th) {
    float mnx = INFINITY, mxx = -INFINITY, mny = INFINITY, mxy = -INFINITY;
    for (int j = -1; j <= 1; ++j)
        for (int k = -1; k <= 1; ++k) {
            int yy = y + j, xx = x + k;
            if (yy < 0 || yy >= ty || xx < 0 || xx >= tx) continue;
            float2 v = HMFSR_LD(mv + (size_t)yy * tx + xx);
            mnx = fminf(mnx, v.x); mxx = fmaxf(mxx, v.x);
            mny = fminf(mny, v.y); mxy = fmaxf(mxy, v.y);
        }
    double Mx = __dsub_rn((double)mxx, (double)mnx), My = __dsub_rn((double)mxy, (double)mny);
    return length_exceeds(__dadd_rn(__dmul_rn(Mx, Mx), __dmul_rn(My, My)), m_th);
}

__device__ __forceinline__ void strength(const float2 *__restrict__ motion, int n, int ty, int tx, float m_th, float s1,
                                         float s2, float *__restrict__ s_tile, int i) {
    if (i >= n * ty * tx) return;
    int f = i / (ty * tx), r = i % (ty * tx), y = r / tx, x = r % tx;
    HMFSR_ST(s_tile + i, motion_span_exceeds(motion + (size_t)f * ty * tx, ty, tx, y, x, m_th) ? s1 : s2);
}

// --------------------------------------------------------------------------------------
// high-frequency artifact test (supplement, High Frequency Artifacts Removal) of base
// texel (u, v): the 3x3 local means keep less than kappa of the local variance.  With
// the green guide at half scale, 4 x the two variances times 81 and 6561 are the exact
// integers B = sum_c w_c (9 S2 - S1^2) at the texel and A = sum_c w_c (9 sum_k S1_k^2 -
// (sum_k S1_k)^2) over its 3x3 texels (clamped to the grid), w = (4, 1, 4); the test
// A < kappa 81 B is taken in FP64 from exact integers, as a CPU restatement takes it.
// --------------------------------------------------------------------------------------
__device__ __forceinline__ void hf_flag_px(const uint16_t *__restrict__ burst, const uint2 *__restrict__ s1,
                                           const Geom &g, float kappa, unsigned char *__restrict__ flag, int u, int v) {
    if (u >= g.wh || v >= g.hh) return;
    const uint16_t *fr = burst + (size_t)g.ref * g.h * g.pitch;
    const uint2 *S = s1 + (size_t)g.ref * g.hh * g.wh;
    long long sq[3] = {0, 0, 0};  // 3x3 sums of squared guide values at (u, v)
    for (int j = -1; j <= 1; ++j)
        for (int i = -1; i <= 1; ++i) {
            const uint16_t *q = fr + (size_t)(2 * clampi(v + j, 0, g.hh - 1)) * g.pitch + 2 * clampi(u + i, 0, g.wh - 1);
            const uint32_t a = HMFSR_LDG(reinterpret_cast<const uint32_t *>(q));
            const uint32_t b = HMFSR_LDG(reinterpret_cast<const uint32_t *>(q + g.pitch));
            const long long R = a & 0xffffu, G = (a >> 16) + (b & 0xffffu), B = b >> 16;
            sq[0] += R * R; sq[1] += G * G; sq[2] += B * B;
        }
    long long t1[3] = {0, 0, 0}, t2[3] = {0, 0, 0}, c1[3] = {0, 0, 0};
    for (int j = -1; j <= 1; ++j)
        for (int i = -1; i <= 1; ++i) {
            const uint2 m = HMFSR_LDG(S + (size_t)clampi(v + j, 0, g.hh - 1) * g.wh + clampi(u + i, 0, g.wh - 1));
            const long long k[3] = {(long long)(m.x & 0xffffu), (long long)m.y, (long long)(m.x >> 16)};
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                t1[c] += k[c];
                t2[c] += k[c] * k[c];
                if (i == 0 && j == 0) c1[c] = k[c];
            }
        }
    const long long wgt[3] = {4, 1, 4};
    long long A = 0, B = 0;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        B += wgt[c] * (9 * sq[c] - c1[c] * c1[c]);
        A += wgt[c] * (9 * t2[c] - t1[c] * t1[c]);
    }
    HMFSR_ST(flag + (size_t)v * g.wh + u,
             (unsigned char)((B > 0 && (double)A < __dmul_rn((double)kappa, __dmul_rn(81.0, (double)B))) ? 1 : 0));
}

// --------------------------------------------------------------------------------------
// robustness (Eq. 5, 6) and its 5x5 minimum (Eq. 9) on one strip of base texels of one
// frame: one warp, kRobOut columns, `rows` rows.  Each lane evaluates R at two texel
// columns for the rows v0 - 2 .. v0 + rows + 1, walking down: within a motion tile the
// bilinear neighbours of the row below are the bottom neighbours of this row, so each row
// reads new sums for the bottom neighbours only.  A rolling window of five row minima
// gives the column minimum.  Every lane of the warp calls this.
// --------------------------------------------------------------------------------------
constexpr int kRobStrip = 64;  // default strip height, as for kPrepStrip
constexpr float kLog2e = 1.44269504088896340736f;

// Wiener-shrunk squared difference of one channel (Eq. 6): (d d^2 / (d^2 + dmd^2))^2 added
// to dd; a zero denominator means a zero difference
__device__ __forceinline__ float wiener_add(float d, float dmd2, float dd) {
    const float d2 = d * d;
    const float w = (d * d2) * fast_rcp(fmaxf(d2 + dmd2, 1e-30f));
    return fmaf(w, w, dd);
}

// --------------------------------------------------------------------------------------
// Lane l of a warp owns texel columns u0 - 2 + 2 l and u0 - 1 + 2 l (u0 even, so both lie
// in one motion tile); the warp writes the kRobOut columns u0 .. u0 + kRobOut - 1 (lanes
// 1 .. 30).  The pair shares the middle column of its bilinear neighbours (three per row),
// the loop and tile bookkeeping, and a 5-wide row minimum built from the two neighbouring
// lanes' pairs.  The guide sums become floats exactly (a 16- or 17-bit value in the
// mantissa of 2^23, minus 2^23), so every difference base - neighbour is exact, as an
// integer difference would be.
// --------------------------------------------------------------------------------------
constexpr int kRobOut = 60;

// exact float of 0 <= v < 2^23
__device__ __forceinline__ float small_uint_to_float(uint32_t v) { return __uint_as_float(0x4B000000u | v) - 8388608.f; }

struct GuideSums {
    float r, b, g;
};
__device__ __forceinline__ GuideSums guide_sums(uint2 s) {
    return {small_uint_to_float(s.x & 0xffffu), small_uint_to_float(s.x >> 16), small_uint_to_float(s.y)};
}

// R of one texel (Eq. 5, 6) from its base sums and the four bilinear neighbours' sums
// (top-left, top-right, bottom-left, bottom-right) with weights b00 .. b11
__device__ __forceinline__ float rob_texel(const GuideSums &s, const GuideSums &n00, const GuideSums &n10,
                                           const GuideSums &n01, const GuideSums &n11, float b00, float b10, float b01,
                                           float b11, const float4 &st, float sc, float t_thr) {
    float dR = fmaf(b00, s.r - n00.r, fmaf(b10, s.r - n10.r, fmaf(b01, s.r - n01.r, b11 * (s.r - n11.r))));
    float dB = fmaf(b00, s.b - n00.b, fmaf(b10, s.b - n10.b, fmaf(b01, s.b - n01.b, b11 * (s.b - n11.b))));
    float dG = fmaf(b00, s.g - n00.g, fmaf(b10, s.g - n10.g, fmaf(b01, s.g - n01.g, b11 * (s.g - n11.g))));
    dR *= (1.f / 9.f);
    dB *= (1.f / 9.f);
    dG *= (1.f / 18.f);
    const float dd = wiener_add(dB, st.w, wiener_add(dG, st.z, wiener_add(dR, st.y, 0.f)));
    const float ex = fast_exp2(-(dd * fast_rcp(st.x)) * kLog2e);
    return fminf(fmaxf(fmaf(sc, ex, -t_thr), 0.f), 1.f);
}

// kHF: hf_flag holds the base texels' high-frequency flags, which reject (R = 0) where
// the tile's motion span exceeds m_th (otherwise both are unused)
template <bool kHF = false>
__device__ __forceinline__ void rob_strip(const uint2 *__restrict__ s1, const float4 *__restrict__ base_stats,
                                           const float2 *__restrict__ motion, const float *__restrict__ s_tile,
                                           const Geom &g, float t_thr, float *__restrict__ rhat, int u0, int v0,
                                           int frame, int lane, const unsigned char *__restrict__ hf_flag = nullptr,
                                           float m_th = 0.f, int rows = kRobStrip) {
    const size_t hw = (size_t)g.hh * g.wh;
    const int wh = g.wh, ua = u0 - 2 + 2 * lane;
    const bool ok_a = ua >= 0 && ua < wh, ok_b = ua + 1 >= 0 && ua + 1 < wh;
    const int uc = clampi(ua, 0, wh - 1);
    const int ht = g.tile / 2;  // motion tile in texels (even)
    const int txi = min(uc / ht, g.tx - 1);
    const uint2 *S1b = s1 + (size_t)g.ref * hw;
    const uint2 *S1n = s1 + (size_t)frame * hw;
    const float2 *mvf = motion + (size_t)frame * g.ty * g.tx + txi;
    const float *stf = s_tile + (size_t)frame * g.ty * g.tx + txi;
    float *out = rhat + (size_t)frame * hw;
    const int vfirst = max(v0 - 2, 0);
    int tq = vfirst / ht, tr = vfirst - tq * ht;
    int cur_tile = -1, fly = 0, x0 = 0, x1 = 0, x2 = 0;
    bool span = false;
    float b00 = 0.f, b10 = 0.f, b01 = 0.f, b11 = 0.f, sc = 0.f;
    GuideSums t0{}, t1{}, t2{}, n0{}, n1{}, n2{};  // sums at the top / bottom neighbours x0, x1, x2
    bool have_prev = false;
    float ha[4] = {kBig, kBig, kBig, kBig}, hb[4] = {kBig, kBig, kBig, kBig};  // row minima of the rows above
    int off = (v0 - 2) * wh + uc;  // texel a's offset in the row (32-bit offsets)
    for (int e = 0; e < rows + 4; ++e, off += wh) {
        const int v = v0 - 2 + e;
        float ra = kBig, rb = kBig;
        if (v >= 0 && v < g.hh) {  // the same for the whole warp
            const int tyi = min(tq, g.ty - 1);
            if (tyi != cur_tile) {
                cur_tile = tyi;
                const float2 mv = HMFSR_LD(mvf + tyi * g.tx);
                sc = HMFSR_LD(stf + tyi * g.tx);
                const float hx = 0.5f * mv.x, hy = 0.5f * mv.y;
                const float flx = floorf(hx), flyf = floorf(hy);
                const float fx = hx - flx, fy = hy - flyf;
                b00 = (1.f - fx) * (1.f - fy); b10 = fx * (1.f - fy); b01 = (1.f - fx) * fy; b11 = fx * fy;
                fly = (int)flyf;
                x0 = clampi(uc + (int)flx, 0, wh - 1);
                x1 = clampi(uc + (int)flx + 1, 0, wh - 1);
                x2 = clampi(uc + (int)flx + 2, 0, wh - 1);
                have_prev = false;
                if (kHF) span = motion_span_exceeds(motion + (size_t)frame * g.ty * g.tx, g.ty, g.tx, tyi, txi, m_th);
            }
            if (++tr == ht) { tr = 0; ++tq; }
            const int iy = v + fly;
            if (have_prev) {
                t0 = n0; t1 = n1; t2 = n2;
            } else {
                const int o0 = clampi(iy, 0, g.hh - 1) * wh;
                t0 = guide_sums(HMFSR_LD(S1n + o0 + x0));
                t1 = guide_sums(HMFSR_LD(S1n + o0 + x1));
                t2 = guide_sums(HMFSR_LD(S1n + o0 + x2));
            }
            const int o1 = clampi(iy + 1, 0, g.hh - 1) * wh;
            n0 = guide_sums(HMFSR_LD(S1n + o1 + x0));
            n1 = guide_sums(HMFSR_LD(S1n + o1 + x1));
            n2 = guide_sums(HMFSR_LD(S1n + o1 + x2));
            have_prev = true;
            if (ok_a) {
                if (kHF && span && HMFSR_LD(hf_flag + off)) ra = 0.f;
                else ra = rob_texel(guide_sums(HMFSR_LD(S1b + off)), t0, t1, n0, n1, b00, b10, b01, b11,
                                    HMFSR_LD(base_stats + off), sc, t_thr);
            }
            if (ok_b) {
                if (kHF && span && HMFSR_LD(hf_flag + off + 1)) rb = 0.f;
                else rb = rob_texel(guide_sums(HMFSR_LD(S1b + off + 1)), t1, t2, n1, n2, b00, b10, b01, b11,
                                    HMFSR_LD(base_stats + off + 1), sc, t_thr);
            }
        } else {
            have_prev = false;
        }
        // 5-wide row minima: the previous lane's pair, this pair, the next lane's pair
        const float pa = __shfl_up_sync(0xffffffffu, ra, 1), pb = __shfl_up_sync(0xffffffffu, rb, 1);
        const float na = __shfl_down_sync(0xffffffffu, ra, 1), nb = __shfl_down_sync(0xffffffffu, rb, 1);
        const float mid = fminf(ra, rb);
        const float ma = fminf(fminf(pa, pb), fminf(mid, na));
        const float mb = fminf(fminf(pb, mid), fminf(na, nb));
        if (e >= 4 && lane >= 1 && lane <= 30) {
            const int vo = v - 2;
            if (vo < g.hh) {
                if (ua < wh) HMFSR_ST(out + vo * wh + ua, fminf(fminf(fminf(ha[0], ha[1]), fminf(ha[2], ha[3])), ma));
                if (ua + 1 < wh)
                    HMFSR_ST(out + vo * wh + ua + 1, fminf(fminf(fminf(hb[0], hb[1]), fminf(hb[2], hb[3])), mb));
            }
        }
        ha[0] = ha[1]; ha[1] = ha[2]; ha[2] = ha[3]; ha[3] = ma;
        hb[0] = hb[1]; hb[1] = hb[2]; hb[2] = hb[3]; hb[3] = mb;
    }
}

}  // namespace stage
}  // namespace hmfsr
