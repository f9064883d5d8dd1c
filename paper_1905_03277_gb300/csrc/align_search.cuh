// Tile alignment (Sec. 3.2): the block-matching searches, the Lucas-Kanade refinement and
// the quadratic-fit step for one tile size.  Each align_t<T>.cu includes this for one tile
// size, so the many (tile, radius) instantiations compile in parallel translation units.
// The per-item bodies live in stages.cuh, shared with the batched persistent kernel.
#pragma once

#include "stages.cuh"

namespace hmfsr {
namespace {

// Block matching of one tile per block for the coarse levels, where there are few tiles:
// the tile's candidate window and reference are staged in shared memory and thread c of
// the (2 RAD + 1)^2 offsets sums its own candidate, so a tile takes the latency of one
// candidate's sum; the block's minimum key decides (same sums and keys as ssd()).
template <int T, int RAD>
struct TileSsd {
    static constexpr int kW = 2 * RAD + 1, kA = T + 2 * RAD;
    static constexpr int kThreads = ((kW * kW + 31) / 32) * 32;
};

template <int T, int RAD, int PART>
__global__ void __launch_bounds__(TileSsd<T, RAD>::kThreads) k_ssd_tile(const uint16_t *__restrict__ img, int lh,
                                                                        int lw, int lty, int ltx,
                                                                        const int2 *__restrict__ parent, int pty,
                                                                        int ptx, int fsh, int ref,
                                                                        int2 *__restrict__ vec) {
    using S = TileSsd<T, RAD>;
    constexpr int kW = S::kW, kA = S::kA, kNT = S::kThreads, kWarps = kNT / 32;
    __shared__ int win[kA][kA];
    __shared__ int rf[T][T];
    __shared__ unsigned long long wmin[kWarps];
    const int tile = blockIdx.x, f = blockIdx.y, tid = threadIdx.x;
    int2 *out = vec + (size_t)f * lty * ltx + tile;
    if (f == ref) {
        if (tid == 0) HMFSR_ST(out, make_int2(0, 0));
        return;
    }
    const int ty = tile / ltx, tx = tile - ty * ltx;
    const int2 cc = stage::ssd_centre(parent, pty, ptx, fsh, tx, ty, T, f);
    const uint16_t *R = img + (size_t)ref * lh * lw;
    const uint16_t *A = img + (size_t)f * lh * lw;
    const int x0 = tx * T, y0 = ty * T, xa = x0 + cc.x - RAD, ya = y0 + cc.y - RAD;
    for (int k = tid; k < kA * kA; k += kNT) {
        const int r = k / kA, c = k - r * kA;
        win[r][c] = HMFSR_LDG(A + (size_t)clampi(ya + r, 0, lh - 1) * lw + clampi(xa + c, 0, lw - 1));
    }
    for (int k = tid; k < T * T; k += kNT) {
        const int j = k / T, i = k - j * T;
        rf[j][i] = HMFSR_LDG(R + (size_t)min(y0 + j, lh - 1) * lw + clampi(x0 + i, 0, lw - 1));
    }
    __syncthreads();
    unsigned long long key = ~0ull;
    if (tid < kW * kW) {
        const int dyi = tid / kW, dxi = tid - dyi * kW;
        stage::SsdAcc<T, PART> acc;
#pragma unroll 2
        for (int j = 0; j < T; ++j) {
            int rv[T], av[T];
#pragma unroll
            for (int i = 0; i < T; ++i) {
                rv[i] = rf[j][i];
                av[i] = win[j + dyi][i + dxi];
            }
            acc.add(rv, av, j);
        }
        key = stage::ssd_key(acc.total, dxi - RAD, dyi - RAD);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long k2 = __shfl_xor_sync(0xffffffffu, key, o);
        key = k2 < key ? k2 : key;
    }
    if ((tid & 31) == 0) wmin[tid >> 5] = key;
    __syncthreads();
    if (tid == 0) {
        unsigned long long m = wmin[0];
#pragma unroll
        for (int w = 1; w < kWarps; ++w) m = wmin[w] < m ? wmin[w] : m;
        const int bdx = (int)(m & 15ull) - 7, bdy = (int)((m >> 4) & 15ull) - 7;
        HMFSR_ST(out, make_int2(cc.x + bdx, cc.y + bdy));
    }
}

template <int T, int RAD, int PART>
__global__ void __launch_bounds__(64) k_ssd_rows(const uint16_t *__restrict__ img, int lh, int lw, int lty, int ltx,
                                                 const int2 *__restrict__ parent, int pty, int ptx, int fsh, int ref,
                                                 int2 *__restrict__ vec) {
    stage::ssd_rows<T, RAD, PART>(img, lh, lw, lty, ltx, parent, pty, ptx, fsh, ref, vec,
                                  blockIdx.x * blockDim.x + threadIdx.x, blockIdx.y);
}

// 4 warps of 32 / (2 RAD + 1) tiles each
template <int T, int RAD, int PART>
__global__ void __launch_bounds__(128) k_ssd_group(const uint16_t *__restrict__ img, int lh, int lw, int lty, int ltx,
                                                   const int2 *__restrict__ parent, int pty, int ptx, int fsh, int ref,
                                                   int2 *__restrict__ vec) {
    constexpr int kG = 32 / (2 * RAD + 1);
    const int warp = blockIdx.x * 4 + (threadIdx.x >> 5);
    stage::ssd_group<T, RAD, PART>(img, lh, lw, lty, ltx, parent, pty, ptx, fsh, ref, vec, warp * kG,
                                   threadIdx.x & 31, blockIdx.y);
}

// Block matching of one level with each warp's candidate windows staged in shared memory.
// A warp takes kG = 32 / (2 RAD + 1) tiles, as k_ssd_group does (lane d of a group takes
// the offsets dy = d - RAD).  The warp first copies, for each of its tiles, the T + 2 RAD
// candidate rows of T + 2 RAD texels and the tile's T reference rows into shared memory
// (as ints, each row once, through 16-byte loads where the rows allow); every lane then
// reads its rows from there with 16-byte shared loads.  Same sums and keys as ssd_group,
// so the same vectors.
template <int T, int RAD>
struct StagedSsd {
    static constexpr int kW = 2 * RAD + 1, kG = 32 / kW, kA = T + 2 * RAD;
    static constexpr int kS = ((kA + 3) & ~3) + 4;  // window row stride (ints): 16-byte rows, banks spread
    static constexpr int kWin = kA * kS;
    static constexpr int kTile = kWin + T * T;      // ints per tile: window, then the T x T reference
    static constexpr int kWarps = 4;
    static constexpr size_t kBytes = sizeof(int) * kWarps * kG * kTile;
};

template <int T, int RAD, int PART>
__global__ void __launch_bounds__(128) k_ssd_staged(const uint16_t *__restrict__ img, int lh, int lw, int lty, int ltx,
                                                    const int2 *__restrict__ parent, int pty, int ptx, int fsh,
                                                    int ref, int2 *__restrict__ vec) {
    using S = StagedSsd<T, RAD>;
    constexpr int kW = S::kW, kG = S::kG, kA = S::kA, kS = S::kS;
    static_assert(T % 4 == 0 && kS % 4 == 0, "16-byte shared rows");
    __shared__ __align__(16) int sm[S::kWarps][kG][S::kTile];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, f = blockIdx.y;
    const int tile0 = (blockIdx.x * S::kWarps + warp) * kG, ntiles = lty * ltx;
    const int grp = lane / kW, d = lane - grp * kW;
    const int tile = tile0 + grp;
    const bool active = grp < kG && tile < ntiles;
    if (f == ref) {
        if (active && d == 0) HMFSR_ST(vec + (size_t)f * ntiles + tile, make_int2(0, 0));
        return;
    }
    const uint16_t *R = img + (size_t)ref * lh * lw;
    const uint16_t *A = img + (size_t)f * lh * lw;
    const bool al16 = stage::rows_aligned16(img, lw);
    // candidate rows: kG x kA rows over the warp's lanes
    for (int r = lane; r < kG * kA; r += 32) {
        const int g = r / kA, rr = r - g * kA, t = tile0 + g;
        if (t >= ntiles) continue;
        const int ty = t / ltx, tx = t - ty * ltx;
        const int2 cc = stage::ssd_centre(parent, pty, ptx, fsh, tx, ty, T, f);
        const int x0 = tx * T, y0 = ty * T, xa = x0 + cc.x - RAD;
        const bool inside = stage::ssd_inside(x0, xa, T, RAD, lw);
        int v[kA];
        stage::load_row2(A + (size_t)clampi(y0 + cc.y - RAD + rr, 0, lh - 1) * lw, xa, lw, inside, inside && al16, v);
        int4 *dst = reinterpret_cast<int4 *>(&sm[warp][g][rr * kS]);
#pragma unroll
        for (int i = 0; i < kA / 4; ++i) dst[i] = make_int4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
        if constexpr (kA % 4 != 0) {
#pragma unroll
            for (int i = kA & ~3; i < kA; ++i) sm[warp][g][rr * kS + i] = v[i];
        }
    }
    // reference rows: kG x T rows
    for (int r = lane; r < kG * T; r += 32) {
        const int g = r / T, j = r - g * T, t = tile0 + g;
        if (t >= ntiles) continue;
        const int ty = t / ltx, tx = t - ty * ltx;
        const int x0 = tx * T, y0 = ty * T;
        const bool inside = x0 + T <= lw;
        int v[T];
        stage::load_row2<T, T % 8 == 0>(R + (size_t)min(y0 + j, lh - 1) * lw, x0, lw, inside, inside && al16, v);
        int4 *dst = reinterpret_cast<int4 *>(&sm[warp][g][S::kWin + j * T]);
#pragma unroll
        for (int i = 0; i < T / 4; ++i) dst[i] = make_int4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
    }
    __syncwarp();
    unsigned long long best = ~0ull;
    if (active) {
        const int *win = &sm[warp][grp][d * kS];  // candidate row j + d of the window at row j
        const int *rf = &sm[warp][grp][S::kWin];
        stage::SsdAcc<T, PART> acc[kW];
#pragma unroll 2
        for (int j = 0; j < T; ++j) {
            int rv[T], av[kA];
            const int4 *pr = reinterpret_cast<const int4 *>(rf + j * T);
            const int4 *pa = reinterpret_cast<const int4 *>(win + j * kS);
#pragma unroll
            for (int i = 0; i < T / 4; ++i) {
                const int4 q = pr[i];
                rv[4 * i] = q.x; rv[4 * i + 1] = q.y; rv[4 * i + 2] = q.z; rv[4 * i + 3] = q.w;
            }
#pragma unroll
            for (int i = 0; i < kA / 4; ++i) {
                const int4 q = pa[i];
                av[4 * i] = q.x; av[4 * i + 1] = q.y; av[4 * i + 2] = q.z; av[4 * i + 3] = q.w;
            }
            if constexpr (kA % 4 != 0) {
#pragma unroll
                for (int i = kA & ~3; i < kA; ++i) av[i] = win[j * kS + i];
            }
#pragma unroll
            for (int k = 0; k < kW; ++k) acc[k].add(rv, av + k, j);
        }
#pragma unroll
        for (int k = 0; k < kW; ++k) {
            const unsigned long long key = stage::ssd_key(acc[k].total, k - RAD, d - RAD);
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
        const int ty = tile / ltx, tx = tile - ty * ltx;
        const int2 cc = stage::ssd_centre(parent, pty, ptx, fsh, tx, ty, T, f);
        const int bdx = (int)(m & 15ull) - 7, bdy = (int)((m >> 4) & 15ull) - 7;
        HMFSR_ST(vec + (size_t)f * ntiles + tile, make_int2(cc.x + bdx, cc.y + bdy));
    }
}

template <int T>
__global__ void __launch_bounds__(128) k_quadfit(const uint16_t *__restrict__ L0, int lh, int lw, int lty, int ltx,
                                                 const int2 *__restrict__ vec0, int ref, float *__restrict__ motion,
                                                 int32_t *__restrict__ motion_int) {
    stage::quadfit<T>(L0, lh, lw, lty, ltx, vec0, ref, motion, motion_int, blockIdx.x * blockDim.x + threadIdx.x,
                      blockIdx.y);
}

template <int T>
__global__ void __launch_bounds__(128, 6) k_lk_group(const uint16_t *__restrict__ L0, int lh, int lw, int lty, int ltx,
                           const int2 *__restrict__ vec0, int ref, int iters, float *__restrict__ motion,
                           int32_t *__restrict__ motion_int) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    stage::lk_group<T>(L0, lh, lw, lty, ltx, vec0, ref, iters, motion, motion_int, t / (T / 2), threadIdx.x & 31,
                       blockIdx.y);
}

// Level 0 searched (radius 1) and refined in one launch: a tile's T / 2 lanes find its
// integer vector (ssd0_lanes), write it to the level-0 vectors, and run Lucas-Kanade from it.
template <int T, int PART>
__global__ void __launch_bounds__(128, 6) k_ssd0_lk(const uint16_t *__restrict__ L0, int lh, int lw, int lty, int ltx,
                                                    const int2 *__restrict__ parent, int pty, int ptx, int fsh,
                                                    int ref, int2 *__restrict__ vec0, int iters,
                                                    float *__restrict__ motion, int32_t *__restrict__ motion_int) {
    constexpr int kL = T / 2;
    const int t = blockIdx.x * blockDim.x + threadIdx.x, lane = threadIdx.x & 31, f = blockIdx.y;
    const int tile = t / kL;
    const bool lead = tile < lty * ltx && (lane & (kL - 1)) == 0;
    const size_t o = (size_t)f * lty * ltx + tile;
    if (f == ref) {
        if (lead) {
            HMFSR_ST(vec0 + o, make_int2(0, 0));
            HMFSR_ST(motion + 2 * o, 0.f);
            HMFSR_ST(motion + 2 * o + 1, 0.f);
            if (motion_int) { HMFSR_ST(motion_int + 2 * o, 0); HMFSR_ST(motion_int + 2 * o + 1, 0); }
        }
        return;
    }
    const int2 u = stage::ssd0_lanes<T, PART>(L0, lh, lw, lty, ltx, parent, pty, ptx, fsh, ref, tile, lane, f);
    if (lead) HMFSR_ST(vec0 + o, u);
    stage::lk_group_u<T>(L0, lh, lw, lty, ltx, ref, iters, motion, motion_int, tile, lane, f, u);
}

template <int T>
__global__ void k_lk(const uint16_t *__restrict__ L0, int lh, int lw, int lty, int ltx, const int2 *__restrict__ vec0,
                     int ref, int iters, float *__restrict__ motion, int32_t *__restrict__ motion_int) {
    stage::lk<T>(L0, lh, lw, lty, ltx, vec0, ref, iters, motion, motion_int,
                 (blockIdx.x * blockDim.x + threadIdx.x) >> 5, threadIdx.x & 31, blockIdx.y);
}

}  // namespace

// Block matching of one level: rows outermost for small radii and tiles, else the offsets
// dy spread over the lanes of a group (measured at 12 MP on level 1, 96k tile-frames: the
// grouped form 9 us faster than one thread per tile, both at 64 registers).

// at most this many tile-frames: a level is searched one tile per block (k_ssd_tile)
constexpr long long kTileSearchMax = 16384;

template <int T, int RAD, int PART>
static void launch_ssd_part(const AlignLevels &L, int l, int n, int ref, int fsh, bool top, cudaStream_t s) {
    const int tiles = L.lty[l] * L.ltx[l];
    const int2 *parent = top ? nullptr : L.vec[l + 1];
    const int pty = top ? 0 : L.lty[l + 1], ptx = top ? 0 : L.ltx[l + 1];
    if (RAD >= 2 && (long long)tiles * n <= kTileSearchMax) {
        k_ssd_tile<T, RAD, PART><<<dim3(tiles, n), TileSsd<T, RAD>::kThreads, 0, s>>>(
            L.img[l], L.lh[l], L.lw[l], L.lty[l], L.ltx[l], parent, pty, ptx, fsh, ref, L.vec[l]);
    } else if constexpr (RAD <= 2 && T <= 8) {
        k_ssd_rows<T, RAD, PART><<<dim3(div_up(tiles, 64), n), 64, 0, s>>>(
            L.img[l], L.lh[l], L.lw[l], L.lty[l], L.ltx[l], parent, pty, ptx, fsh, ref, L.vec[l]);
    } else if constexpr (T <= 16 && StagedSsd<T, RAD>::kBytes <= 40 * 1024) {
        constexpr int kTilesPerBlock = StagedSsd<T, RAD>::kWarps * StagedSsd<T, RAD>::kG;
        k_ssd_staged<T, RAD, PART><<<dim3(div_up(tiles, kTilesPerBlock), n), 128, 0, s>>>(
            L.img[l], L.lh[l], L.lw[l], L.lty[l], L.ltx[l], parent, pty, ptx, fsh, ref, L.vec[l]);
    } else {
        constexpr int kTilesPerBlock = 4 * (32 / (2 * RAD + 1));
        k_ssd_group<T, RAD, PART><<<dim3(div_up(tiles, kTilesPerBlock), n), 128, 0, s>>>(
            L.img[l], L.lh[l], L.lw[l], L.lty[l], L.ltx[l], parent, pty, ptx, fsh, ref, L.vec[l]);
    }
}

// Level values are at most 4 WL (a level-0 texel sums four samples <= WL; coarser levels
// average): below 2^14 for WL <= 4095, where 16 squared differences fit a 32-bit partial.
template <int T, int RAD>
static void launch_ssd(const AlignLevels &L, int l, int n, int ref, int fsh, bool top, int wl, cudaStream_t s) {
    if (wl <= 4095) launch_ssd_part<T, RAD, 16>(L, l, n, ref, fsh, top, s);
    else launch_ssd_part<T, RAD, 4>(L, l, n, ref, fsh, top, s);
}

template <int T>
static void run_search(const Geom &g, const hmfsr_align_params &p, const AlignLevels &L, float *motion,
                       int32_t *motion_int, cudaStream_t s) {
    static const int kShift[3] = {1, 2, 2};  // log2 of the factors 2, 4, 4
    const int n = g.n;
    // level 0 at radius 1 with tiles of at most 8 texels: searched inside the refinement launch
    const bool fused0 = (T <= 8) && p.radius[0] == 1;
    for (int l = L.n_levels - 1; l >= (fused0 ? 1 : 0); --l) {
        const bool top = (l == L.n_levels - 1);
        const int fsh = top ? 0 : kShift[l];
        switch (p.radius[l]) {
            case 0: launch_ssd<T, 0>(L, l, n, g.ref, fsh, top, g.wl, s); break;
            case 1: launch_ssd<T, 1>(L, l, n, g.ref, fsh, top, g.wl, s); break;
            case 2: launch_ssd<T, 2>(L, l, n, g.ref, fsh, top, g.wl, s); break;
            case 3: launch_ssd<T, 3>(L, l, n, g.ref, fsh, top, g.wl, s); break;
            case 4: launch_ssd<T, 4>(L, l, n, g.ref, fsh, top, g.wl, s); break;
            case 5: launch_ssd<T, 5>(L, l, n, g.ref, fsh, top, g.wl, s); break;
            case 6: launch_ssd<T, 6>(L, l, n, g.ref, fsh, top, g.wl, s); break;
            default: launch_ssd<T, stage::kMaxRad>(L, l, n, g.ref, fsh, top, g.wl, s); break;
        }
    }
    const int tiles0 = L.lty[0] * L.ltx[0];
    if constexpr (T <= 8) {
        if (fused0) {
            const bool top = L.n_levels == 1;
            const int2 *parent = top ? nullptr : L.vec[1];
            const int pty = top ? 0 : L.lty[1], ptx = top ? 0 : L.ltx[1], fsh = top ? 0 : kShift[0];
            const dim3 grid(div_up(tiles0 * (T / 2), 128), n);
            if (g.wl <= 4095)
                k_ssd0_lk<T, 16><<<grid, 128, 0, s>>>(L.img[0], L.lh[0], L.lw[0], L.lty[0], L.ltx[0], parent, pty, ptx,
                                                      fsh, g.ref, L.vec[0], p.lk_iters, motion, motion_int);
            else
                k_ssd0_lk<T, 4><<<grid, 128, 0, s>>>(L.img[0], L.lh[0], L.lw[0], L.lty[0], L.ltx[0], parent, pty, ptx,
                                                     fsh, g.ref, L.vec[0], p.lk_iters, motion, motion_int);
            return;
        }
        k_lk_group<T><<<dim3(div_up(tiles0 * (T / 2), 128), n), 128, 0, s>>>(
            L.img[0], L.lh[0], L.lw[0], L.lty[0], L.ltx[0], L.vec[0], g.ref, p.lk_iters, motion, motion_int);
    } else {
        k_lk<T><<<dim3(div_up(tiles0 * 32, 128), n), 128, 0, s>>>(L.img[0], L.lh[0], L.lw[0], L.lty[0], L.ltx[0],
                                                           L.vec[0], g.ref, p.lk_iters, motion, motion_int);
    }
}

template <int T>
static void launch_quadfit(const Geom &g, const AlignLevels &L, float *motion, int32_t *motion_int, cudaStream_t s) {
    const int tiles0 = L.lty[0] * L.ltx[0];
    k_quadfit<T><<<dim3(div_up(tiles0, 128), g.n), 128, 0, s>>>(L.img[0], L.lh[0], L.lw[0], L.lty[0], L.ltx[0],
                                                               L.vec[0], g.ref, motion, motion_int);
}

// the searches of every level and the refinement, for tiles of T level texels
template <int T>
cudaError_t align_search_tiles(const Geom &g, const hmfsr_align_params &p, const AlignLevels &L, float *motion,
                               int32_t *motion_int, cudaStream_t s) {
    CheckedLaunches checked(s);
    run_search<T>(g, p, L, motion, motion_int, s);
    return cudaGetLastError();
}

// the quadratic-fit subpixel step from the level-0 vectors, for tiles of T level texels
template <int T>
cudaError_t align_quadfit_tiles(const Geom &g, const AlignLevels &L, float *motion, int32_t *motion_int,
                                cudaStream_t s) {
    CheckedLaunches checked(s);
    launch_quadfit<T>(g, L, motion, motion_int, s);
    return cudaGetLastError();
}

}  // namespace hmfsr
