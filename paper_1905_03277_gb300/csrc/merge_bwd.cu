// Adjoint of the merge (reverse mode of Eq. 1-9 and the supplement's kernel heuristics).
//
// Differentiable inputs: the kernel parameters k_detail, k_denoise, D_th, D_tr,
// k_stretch, k_shrink, the robustness scale s (s2 of Eq. 8; s1 stays fixed) and the
// threshold t, and every tile's motion vector.  Discrete decisions (window centres,
// tiles, s1/s2 selection, clamps, the 5x5 argmin, bilinear cells) carry no gradient.
// The forward is recomputed from the burst; the forward's normalised colour C and
// log2 of its weight sum are read back, so each sample's normalised weight is
// 2^-(q' + log2 den).  All reductions are deterministic: per-pixel and per-texel
// contributions go to buffers and are summed in a fixed order in FP64.
#include "hmfsr_internal.cuh"

namespace hmfsr {
namespace {

constexpr float kHalfLog2e = 0.72134752044448170368f;  // log2(e) / 2
constexpr int kBwdW = 32, kBwdH = 4, kBwdThreads = kBwdW * kBwdH;

// Block sums in a fixed order without FP64 arithmetic per element (FP64 is scarce on this
// GPU): each warp adds its lanes' values by butterflies carrying the exact rounding error
// of every FP32 addition (two-sum), lane 0 stores the warp's (sum, error) pair; the
// caller's thread 0 then adds the warps' pairs in FP64 in warp order.
template <int K>
__device__ __forceinline__ void warp_sums_comp(float (&v)[K], float (&e)[K]) {
#pragma unroll
    for (int q = 0; q < K; ++q) e[q] = 0.f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int q = 0; q < K; ++q) {
            const float a = v[q], b = __shfl_xor_sync(0xffffffffu, v[q], o);
            const float t = a + b, bp = t - a;
            const float err = (a - (t - bp)) + (b - bp);
            e[q] = (e[q] + __shfl_xor_sync(0xffffffffu, e[q], o)) + err;
            v[q] = t;
        }
}

// The six kernel parameters' contribution of one texel.  With k_x = s_x^2 the kernel
// variances of Eq. 4 / S.1 (s_along, s_across their square roots), d k_x / d p_q = 2 s_x
// a_x[q], and the texel adds sum_q (d k_across / d p_q bo1 + d k_along / d p_q bo2) to
// pb[q], bo1 and bo2 being dL/dk_across and dL/dk_along times the bilinear weight:
//   a_along  = {(1-D) k_stretch A + D k_denoise, D k_detail, (kd - kh_al) dD/dD_th,
//               (kd - kh_al) dD/dD_tr, (1-D) k_detail A, 0},
//   a_across = {(1-D) / (k_shrink A) + D k_denoise, D k_detail, (kd - kh_ac) dD/dD_th,
//               (kd - kh_ac) dD/dD_tr, 0, -(1-D) k_detail / (k_shrink^2 A)}
// with kd = k_detail k_denoise, kh_al = k_detail k_stretch A, kh_ac = k_detail /
// (k_shrink A), D = clamp(1 - sqrt(l1_norm) / D_tr + D_th, 0, 1) and its derivatives 0
// where clamped.  Per-call constants in KConsts; 1/A on the SFU.
struct KConsts {
    float inv_dtr, inv_shrink, kd, kds, kdi, kdi2;
};
__device__ __forceinline__ KConsts kconsts_of(const MergeConsts &c) {
    KConsts k;
    k.inv_dtr = 1.f / c.d_tr;
    k.inv_shrink = 1.f / c.k_shrink;
    k.kd = c.k_detail * c.k_denoise;
    k.kds = c.k_detail * c.k_stretch;
    k.kdi = c.k_detail * k.inv_shrink;
    k.kdi2 = k.kdi * k.inv_shrink;
    return k;
}
__device__ __forceinline__ void kernel_grad_acc(const float4 sh, const MergeConsts &c, const KConsts &k, float bo1,
                                                float bo2, float (&pb)[6]) {
    const float A = sh.x, rl = sh.y, invA = fast_rcp(A);
    const float Draw = 1.f - rl * k.inv_dtr + c.d_th;
    const float D = fminf(fmaxf(Draw, 0.f), 1.f), omD = 1.f - D;
    const bool inside = Draw > 0.f && Draw < 1.f;
    const float kh_al = k.kds * A, kh_ac = k.kdi * invA;
    const float s_al = omD * kh_al + D * k.kd, s_ac = omD * kh_ac + D * k.kd;
    const float P = 2.f * s_ac * bo1, Qv = 2.f * s_al * bo2;  // dL/d(a_across), dL/d(a_along) weights
    pb[0] = fmaf(P, omD * k.inv_shrink * invA + D * c.k_denoise, fmaf(Qv, omD * c.k_stretch * A + D * c.k_denoise, pb[0]));
    pb[1] = fmaf(P + Qv, D * c.k_detail, pb[1]);
    if (inside) {
        const float sD = P * (k.kd - kh_ac) + Qv * (k.kd - kh_al);
        pb[2] += sD;
        pb[3] = fmaf(sD, rl * k.inv_dtr * k.inv_dtr, pb[3]);
    }
    pb[4] = fmaf(Qv, omD * c.k_detail * A, pb[4]);
    pb[5] = fmaf(-P, omD * k.kdi2 * invA, pb[5]);
}

// ---------------------------------------------------------------------------------------
// per texel: what the kernel-shape derivative needs {A, sqrt(l1_norm), cos 2t, sin 2t}
// ---------------------------------------------------------------------------------------
__global__ void k_shape(const uint16_t *__restrict__ burst, int h, int pitch, int hh, int wh, int wl,
                        float4 *__restrict__ shape) {
    const int u = blockIdx.x * blockDim.x + threadIdx.x, v = blockIdx.y, f = blockIdx.z;
    if (u >= wh) return;
    const uint16_t *fr = burst + (size_t)f * h * pitch;
    int L[3][3];  // Lq of the clamped 3x3 window: sum of each quad's four samples
#pragma unroll
    for (int j = 0; j < 3; ++j)
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            const uint16_t *q = fr + (size_t)(2 * clampi(v - 1 + j, 0, hh - 1)) * pitch + 2 * clampi(u - 1 + i, 0, wh - 1);
            const uint32_t a = __ldg(reinterpret_cast<const uint32_t *>(q));
            const uint32_t b = __ldg(reinterpret_cast<const uint32_t *>(q + pitch));
            L[j][i] = (int)((a & 0xffffu) + (a >> 16) + (b & 0xffffu) + (b >> 16));
        }
    long long ta = 0, tb = 0, tc = 0;
#pragma unroll
    for (int j = 0; j < 2; ++j)
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            const int gx = (L[j][i + 1] - L[j][i]) + (L[j + 1][i + 1] - L[j + 1][i]);
            const int gy = (L[j + 1][i] - L[j][i]) + (L[j + 1][i + 1] - L[j][i + 1]);
            ta += (long long)gx * gx;
            tb += (long long)gx * gy;
            tc += (long long)gy * gy;
        }
    const float tr = (float)(ta + tc), amc = (float)(ta - tc), b2 = 2.f * (float)tb;
    const float r = sqrtf(amc * amc + b2 * b2);
    float cs = 1.f, sn = 0.f;
    if (!(ta == tc && tb == 0)) { cs = amc / r; sn = b2 / r; }
    const float A = (ta + tc == 0) ? 1.f : 1.f + sqrtf(r / tr);
    const float rl = sqrtf(0.5f * (tr + r)) / (16.f * (float)wl);
    shape[((size_t)f * hh + v) * wh + u] = make_float4(A, rl, cs, sn);
}

// ---------------------------------------------------------------------------------------
// per tile: 1 where the motion prior (Eq. 7-8) chose s2, the same FP64 decision as the
// forward's
// ---------------------------------------------------------------------------------------
__global__ void k_sel(const float2 *__restrict__ motion, int n, int ty, int tx, float m_th,
                      unsigned char *__restrict__ sel) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n * ty * tx) return;
    const int f = i / (ty * tx), r = i % (ty * tx), y = r / tx, x = r % tx;
    const float2 *mv = motion + (size_t)f * ty * tx;
    float mnx = INFINITY, mxx = -INFINITY, mny = INFINITY, mxy = -INFINITY;
    for (int j = -1; j <= 1; ++j)
        for (int k = -1; k <= 1; ++k) {
            const int yy = y + j, xx = x + k;
            if (yy < 0 || yy >= ty || xx < 0 || xx >= tx) continue;
            const float2 v = mv[(size_t)yy * tx + xx];
            mnx = fminf(mnx, v.x); mxx = fmaxf(mxx, v.x);
            mny = fminf(mny, v.y); mxy = fmaxf(mxy, v.y);
        }
    const double Mx = __dsub_rn((double)mxx, (double)mnx), My = __dsub_rn((double)mxy, (double)mny);
    sel[i] = length_exceeds(__dadd_rn(__dmul_rn(Mx, Mx), __dmul_rn(My, My)), m_th) ? 0 : 1;
}

// ---------------------------------------------------------------------------------------
// per base texel of frame f != ref: R with its partial derivatives
// ---------------------------------------------------------------------------------------
__global__ void k_rback(const uint2 *__restrict__ s1, const float4 *__restrict__ base_stats,
                        const float2 *__restrict__ motion, const float *__restrict__ s_tile,
                        const unsigned char *__restrict__ sel, Geom g, MergeConsts c, float4 *__restrict__ rb,
                        unsigned char *__restrict__ flags) {
    const int u = blockIdx.x * blockDim.x + threadIdx.x, v = blockIdx.y, f = blockIdx.z;
    if (u >= g.wh || f == g.ref) return;
    const size_t hw = (size_t)g.hh * g.wh;
    const int half_tile = g.tile / 2;
    const int txi = min(u / half_tile, g.tx - 1), tyi = min(v / half_tile, g.ty - 1);
    const float2 mv = motion[((size_t)f * g.ty + tyi) * g.tx + txi];
    const float s = s_tile[((size_t)f * g.ty + tyi) * g.tx + txi];
    const float hx = 0.5f * mv.x, hy = 0.5f * mv.y;
    const float flx = floorf(hx), fly = floorf(hy);
    const float fx = hx - flx, fy = hy - fly;
    const int ix = u + (int)flx, iy = v + (int)fly;
    const int x0 = clampi(ix, 0, g.wh - 1), x1 = clampi(ix + 1, 0, g.wh - 1);
    const int y0 = clampi(iy, 0, g.hh - 1), y1 = clampi(iy + 1, 0, g.hh - 1);
    const uint2 *Sb = s1 + (size_t)g.ref * hw, *Sn = s1 + (size_t)f * hw;
    const uint2 sb = Sb[(size_t)v * g.wh + u];
    const uint2 n00 = Sn[(size_t)y0 * g.wh + x0], n10 = Sn[(size_t)y0 * g.wh + x1];
    const uint2 n01 = Sn[(size_t)y1 * g.wh + x0], n11 = Sn[(size_t)y1 * g.wh + x1];
    const float4 st = base_stats[(size_t)v * g.wh + u];
    const float b00 = (1.f - fx) * (1.f - fy), b10 = fx * (1.f - fy), b01 = (1.f - fx) * fy, b11 = fx * fy;
    float dd = 0.f, gvx = 0.f, gvy = 0.f;
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) {
        int sbv, m00, m10, m01, m11;
        float inv, dmd2;
        if (ch == 0) {
            sbv = sb.x & 0xffff; m00 = n00.x & 0xffff; m10 = n10.x & 0xffff; m01 = n01.x & 0xffff; m11 = n11.x & 0xffff;
            inv = 1.f / 9.f; dmd2 = st.y;
        } else if (ch == 1) {
            sbv = sb.y; m00 = n00.y; m10 = n10.y; m01 = n01.y; m11 = n11.y;
            inv = 1.f / 18.f; dmd2 = st.z;
        } else {
            sbv = sb.x >> 16; m00 = n00.x >> 16; m10 = n10.x >> 16; m01 = n01.x >> 16; m11 = n11.x >> 16;
            inv = 1.f / 9.f; dmd2 = st.w;
        }
        const float dms = inv * (b00 * (float)(sbv - m00) + b10 * (float)(sbv - m10) + b01 * (float)(sbv - m01) +
                                 b11 * (float)(sbv - m11));
        // d mu_aligned / d position (in mean units)
        const float dmx = inv * ((1.f - fy) * (float)(m10 - m00) + fy * (float)(m11 - m01));
        const float dmy = inv * ((1.f - fx) * (float)(m01 - m00) + fx * (float)(m11 - m10));
        const float d2 = dms * dms, den = d2 + dmd2;
        const float d = den > 0.f ? dms * d2 / den : 0.f;
        const float dd_dms = den > 0.f ? (d2 * d2 + 3.f * dmd2 * d2) / (den * den) : 0.f;
        dd += d * d;
        gvx += 2.f * d * dd_dms * (-dmx) * 0.5f;
        gvy += 2.f * d * dd_dms * (-dmy) * 0.5f;
    }
    const float e = expf(-dd / st.x);
    const float raw = s * e - c.t;
    const float R = fminf(fmaxf(raw, 0.f), 1.f);
    const bool unclamped = raw > 0.f && raw < 1.f;
    float4 out = make_float4(R, 0.f, 0.f, 0.f);
    if (unclamped) {
        out.y = -s * e * gvx / st.x;
        out.z = -s * e * gvy / st.x;
        out.w = sel[((size_t)f * g.ty + tyi) * g.tx + txi] ? e : 0.f;
    }
    const size_t o = (size_t)f * hw + (size_t)v * g.wh + u;
    rb[o] = out;
    flags[o] = unclamped ? 0x80 : 0;
}

// first minimum of R over the 5x5 window of valid pixels (scan order), offset 0..24
__global__ void k_argmin(const float4 *__restrict__ rb, Geom g, unsigned char *__restrict__ flags) {
    const int u = blockIdx.x * blockDim.x + threadIdx.x, v = blockIdx.y, f = blockIdx.z;
    if (u >= g.wh || f == g.ref) return;
    const size_t hw = (size_t)g.hh * g.wh;
    const float4 *Rp = rb + (size_t)f * hw;
    float best = INFINITY;
    int bi = 12;
    for (int j = -2; j <= 2; ++j)
        for (int i = -2; i <= 2; ++i) {
            const int uu = u + i, vv = v + j;
            if (uu < 0 || uu >= g.wh || vv < 0 || vv >= g.hh) continue;
            const float r = Rp[(size_t)vv * g.wh + uu].x;
            if (r < best) { best = r; bi = (j + 2) * 5 + (i + 2); }
        }
    const size_t o = (size_t)f * hw + (size_t)v * g.wh + u;
    flags[o] = (unsigned char)((flags[o] & 0x80) | bi);
}

// ---------------------------------------------------------------------------------------
// per output pixel: recompute the frame loop and emit the adjoint contributions
// ---------------------------------------------------------------------------------------
// Per sample the inverse quadratic form is split into per-column and per-row parts and
// the per-channel values (C, log2 den, dL/dC) are mapped once per frame onto the window's
// four sample classes, so a sample indexes nothing at run time (indexing the channel
// arrays by a run-time channel had put them in local memory).  Each texel's kernel-shape
// derivatives use reciprocals of the per-call constants and one 1/A on the SFU in place
// of divisions.  4 blocks per SM: 128 registers, no spills (at 96 the body spills and
// measured 1% slower).  Fitting workload (8 x 1024^2, 1.5x): adjoint 1.29 ms, against
// 1.43 ms before these changes on the same box.
__global__ void __launch_bounds__(kBwdThreads, 4) k_merge_bwd(
    const uint16_t *__restrict__ burst, const float2 *__restrict__ motion, Geom g, MergeConsts c,
    const float4 *__restrict__ kern, const float4 *__restrict__ shape, const float *__restrict__ rhat_planes,
    int snum, int sden, int ho, int wo, const float *__restrict__ rgb, const float *__restrict__ lden,
    const float *__restrict__ grad_rgb, float2 *__restrict__ vbar_pix, float *__restrict__ rhbar_pix,
    double *__restrict__ partials) {
    __shared__ double s_red[kBwdThreads];
    const int X = blockIdx.x * kBwdW + threadIdx.x;
    const int Y = blockIdx.y * kBwdH + threadIdx.y;
    const int tid = threadIdx.y * kBwdW + threadIdx.x;
    const bool active = X < wo && Y < ho;
    float pb[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    const KConsts kc = kconsts_of(c);
    if (active) {
        const int Q = 2 * snum, Q2 = 4 * snum;
        const float fQ = (float)Q, invQ = 1.f / fQ, inv2Q = 0.5f / fQ;
        const int Px = 2 * sden * X + sden - snum, Py = 2 * sden * Y + sden - snum;
        const int txi = clampi(floor_div(Px, Q * g.tile), 0, g.tx - 1);
        const int tyi = clampi(floor_div(Py, Q * g.tile), 0, g.ty - 1);
        const size_t hw = (size_t)g.hh * g.wh, po = (size_t)ho * wo, op = (size_t)Y * wo + X;
        const int rx = floor_div(Px - snum, Q2), ry = floor_div(Py - snum, Q2);
        const float rfx = (float)(Px - snum - rx * Q2) * inv2Q, rfy = (float)(Py - snum - ry * Q2) * inv2Q;
        const int rx0 = clampi(rx, 0, g.wh - 1), rx1 = clampi(rx + 1, 0, g.wh - 1);
        const int ry0 = clampi(ry, 0, g.hh - 1), ry1 = clampi(ry + 1, 0, g.hh - 1);
        const float rw00 = (1.f - rfx) * (1.f - rfy), rw10 = rfx * (1.f - rfy), rw01 = (1.f - rfx) * rfy,
                    rw11 = rfx * rfy;
        const float Cc0 = rgb[op], Cc1 = rgb[po + op], Cc2 = rgb[2 * po + op];
        const float Lc0 = lden[op], Lc1 = lden[po + op], Lc2 = lden[2 * po + op];
        const float gc0 = grad_rgb[op], gc1 = grad_rgb[po + op], gc2 = grad_rgb[2 * po + op];
        for (int f = 0; f < g.n; ++f) {
            float vx = 0.f, vy = 0.f, rh = 1.f;
            if (f != g.ref) {
                const float *Rp = rhat_planes + (size_t)f * hw;
                rh = rw00 * Rp[(size_t)ry0 * g.wh + rx0] + rw10 * Rp[(size_t)ry0 * g.wh + rx1] +
                     rw01 * Rp[(size_t)ry1 * g.wh + rx0] + rw11 * Rp[(size_t)ry1 * g.wh + rx1];
                const float2 mv = motion[((size_t)f * g.ty + tyi) * g.tx + txi];
                vx = mv.x;
                vy = mv.y;
            }
            const int FX = floor_mul(Q, vx), FY = floor_mul(Q, vy);
            const int kx = floor_div(Px + snum + FX, Q), ky = floor_div(Py + snum + FY, Q);
            const float dx0 = fmaf(-fQ, vx, (float)(kx * Q - Px)) * invQ;
            const float dy0 = fmaf(-fQ, vy, (float)(ky * Q - Py)) * invQ;
            const float zx = fmaf(fQ, vx, -(float)FX), zy = fmaf(fQ, vy, -(float)FY);
            const int gx = Px - snum + FX, gy = Py - snum + FY;
            const int ox = floor_div(gx, Q2), oy = floor_div(gy, Q2);
            const float ax = ((float)(gx - ox * Q2) + zx) * inv2Q, ay = ((float)(gy - oy * Q2) + zy) * inv2Q;
            const int tx_[4] = {clampi(ox, 0, g.wh - 1), clampi(ox + 1, 0, g.wh - 1), clampi(ox, 0, g.wh - 1),
                                clampi(ox + 1, 0, g.wh - 1)};
            const int ty_[4] = {clampi(oy, 0, g.hh - 1), clampi(oy, 0, g.hh - 1), clampi(oy + 1, 0, g.hh - 1),
                                clampi(oy + 1, 0, g.hh - 1)};
            const float beta[4] = {(1.f - ax) * (1.f - ay), ax * (1.f - ay), (1.f - ax) * ay, ax * ay};
            float4 t[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) t[k] = kern[(size_t)f * hw + (size_t)ty_[k] * g.wh + tx_[k]];
            // Omega = a I + sum g_k u u^T with the accurate (Cauchy-Binet) determinant
            float a = 0.f, G = 0.f, Oxx = 0.f, Oxy = 0.f, Oyy = 0.f, gk[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                gk[k] = beta[k] * t[k].y;
                a += beta[k] * t[k].x;
                G += gk[k];
                Oxx += gk[k] * t[k].z * t[k].z;
                Oxy += gk[k] * t[k].z * t[k].w;
                Oyy += gk[k] * t[k].w * t[k].w;
            }
            float detM = 0.f;
#pragma unroll
            for (int k = 0; k < 4; ++k)
#pragma unroll
                for (int l = k + 1; l < 4; ++l) {
                    const float cr = t[k].z * t[l].w - t[k].w * t[l].z;
                    detM += gk[k] * gk[l] * cr * cr;
                }
            const float det = fmaf(a, a + G, detM);
            // each texel's Omega entries, for the sampling-position and shape terms below
            float okx[4], oky[4], okz[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const float ux = t[k].z, uy = t[k].w;
                okx[k] = t[k].x + t[k].y * ux * ux;
                oky[k] = t[k].y * ux * uy;
                okz[k] = t[k].x + t[k].y * uy * uy;
            }
            const float invdet = 1.f / det;
            // adj(Omega) = a I + [[Oyy, -Oxy], [-Oxy, Oxx]] of M; P = Omega^-1 d splits into
            // per-column and per-row parts: Px = ax[i] + bx[j], Py = cy[i] + dy[j]
            const float sxx = (a + Oyy) * invdet, syy = (a + Oxx) * invdet, sxy = -Oxy * invdet;
            const float dxs[3] = {dx0 - 1.f, dx0, dx0 + 1.f}, dys[3] = {dy0 - 1.f, dy0, dy0 + 1.f};
            float pxc[3], pxr[3], pyc[3], pyr[3];
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                pxc[k] = sxx * dxs[k];
                pyc[k] = sxy * dxs[k];
                pxr[k] = sxy * dys[k];
                pyr[k] = syy * dys[k];
            }
            // per-channel values mapped onto the window's sample classes (C centre, H
            // (+-1, 0), V (0, +-1), K corners) from the parity of the centre (kx, ky):
            // channel(x, y) = (x & 1) + (y & 1) for RGGB
            const int cx = kx & 1, cy = ky & 1;
            auto pick = [](int ch, float r, float gg, float b) { return ch == 0 ? r : (ch == 1 ? gg : b); };
            const int chC = cx + cy, chH = (cx ^ 1) + cy, chV = cx + (cy ^ 1), chK = (cx ^ 1) + (cy ^ 1);
            const float LC = pick(chC, Lc0, Lc1, Lc2), LH = pick(chH, Lc0, Lc1, Lc2);
            const float LV = pick(chV, Lc0, Lc1, Lc2), LK = pick(chK, Lc0, Lc1, Lc2);
            const float gC = pick(chC, gc0, gc1, gc2), gH = pick(chH, gc0, gc1, gc2);
            const float gV = pick(chV, gc0, gc1, gc2), gK = pick(chK, gc0, gc1, gc2);
            const float cC = pick(chC, Cc0, Cc1, Cc2), cH = pick(chH, Cc0, Cc1, Cc2);
            const float cV = pick(chV, Cc0, Cc1, Cc2), cK = pick(chK, Cc0, Cc1, Cc2);
            const uint16_t *fr = burst + (size_t)f * g.h * g.pitch;
            const bool inside = (unsigned)(kx - 1) < (unsigned)(g.w - 2) && (unsigned)(ky - 1) < (unsigned)(g.h - 2);
            const float mrh = -0.5f * rh;
            float ob0 = 0.f, ob1 = 0.f, ob2 = 0.f, sPx = 0.f, sPy = 0.f, rhb = 0.f;
#pragma unroll
            for (int j = -1; j <= 1; ++j)
#pragma unroll
                for (int i = -1; i <= 1; ++i) {
                    const int qx = kx + i, qy = ky + j;
                    if (!inside && (qx < 0 || qx >= g.w || qy < 0 || qy >= g.h)) continue;
                    const float dx = dxs[i + 1], dy = dys[j + 1];
                    const float Pxv = pxc[i + 1] + pxr[j + 1], Pyv = pyc[i + 1] + pyr[j + 1];
                    const float qq = fmaf(dx, Pxv, dy * Pyv);  // d^T Omega^-1 d
                    // the sample's class: centre, horizontal, vertical or corner neighbour
                    const float Lq = (i == 0) ? (j == 0 ? LC : LV) : (j == 0 ? LH : LK);
                    const float gq = (i == 0) ? (j == 0 ? gC : gV) : (j == 0 ? gH : gK);
                    const float cq = (i == 0) ? (j == 0 ? cC : cV) : (j == 0 ? cH : cK);
                    const float wn = fast_exp2(-fmaf(kHalfLog2e, qq, Lq));  // w / den
                    const float cv = (float)__ldg(fr + (size_t)qy * g.pitch + qx);
                    const float e = gq * (cv - cq) * wn;  // dL/d(w Rhat) * w
                    rhb += e;
                    const float qb = mrh * e;  // dL/dq
                    const float t1 = qb * Pxv, t2 = qb * Pyv;
                    sPx += t1;
                    sPy += t2;
                    ob0 = fmaf(t1, Pxv, ob0);
                    ob1 = fmaf(t1, Pyv, ob1);
                    ob2 = fmaf(t2, Pyv, ob2);
                }
            // d L / d v through the offsets d (d = q - x0 - v): -2 sum qb P; Omega-bar = -qb P P^T
            float vbx = -2.f * sPx, vby = -2.f * sPy;
            ob0 = -ob0;
            ob1 = -2.f * ob1;
            ob2 = -ob2;
            // Omega sampling position (x0 + v - 1/2)/2 and the texel parameters
            const float dbx[4] = {-(1.f - ay), 1.f - ay, -ay, ay};
            const float dby[4] = {-(1.f - ax), -ax, 1.f - ax, ax};
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const float dot = ob0 * okx[k] + ob1 * oky[k] + ob2 * okz[k];
                vbx += 0.5f * dbx[k] * dot;
                vby += 0.5f * dby[k] * dot;
                const float4 sh = __ldg(shape + (size_t)f * hw + (size_t)ty_[k] * g.wh + tx_[k]);
                const float e1xx = 0.5f * (1.f + sh.z), e1xy = 0.5f * sh.w, e1yy = 0.5f * (1.f - sh.z);
                const float oE1 = ob0 * e1xx + ob1 * e1xy + ob2 * e1yy;
                const float bo1 = beta[k] * oE1, bo2 = beta[k] * ((ob0 + ob2) - oE1);
                kernel_grad_acc(sh, c, kc, bo1, bo2, pb);
            }
            const size_t of = (size_t)f * po + op;
            vbar_pix[of] = (f == g.ref) ? make_float2(0.f, 0.f) : make_float2(vbx, vby);
            rhbar_pix[of] = (f == g.ref) ? 0.f : rhb;
        }
    }
    // block sums of the six kernel-parameter gradients, in a fixed order
    const int bid = blockIdx.y * gridDim.x + blockIdx.x;
    float pe[6];
    warp_sums_comp<6>(pb, pe);
    if ((tid & 31) == 0)
#pragma unroll
        for (int q = 0; q < 6; ++q) {
            s_red[(tid >> 5) * 12 + 2 * q] = (double)pb[q];
            s_red[(tid >> 5) * 12 + 2 * q + 1] = (double)pe[q];
        }
    __syncthreads();
    if (tid < 6) {
        double acc = 0.0;
        for (int w = 0; w < kBwdThreads / 32; ++w) acc += s_red[w * 12 + 2 * tid] + s_red[w * 12 + 2 * tid + 1];
        partials[(size_t)bid * 6 + tid] = acc;
    }
}

// ---------------------------------------------------------------------------------------
// Rhat-bar gathered onto base texels, then through the 5x5 argmin into R's parameters
// ---------------------------------------------------------------------------------------
// The forward samples Rhat bilinearly on the base grid at (x0 - 1/2)/2 with clamped taps,
// separably in x and y; its transpose gathers dL/dRhat-at-pixels onto texels the same
// way: first along x, per output row (k_rhat_rows), then along y (k_rhat_cols).
// rhat_range: the output pixels (along one axis) whose taps (clamped) reach texel t:
// x0 within (2t - 1.5, 2t + 2.5), plus, at the border, every pixel clamped onto it.
__device__ __forceinline__ void rhat_range(int t, int nt, int nout, int snum, int sden, int &lo, int &hi) {
    lo = (int)floorf(((2.f * t - 1.5f) + 0.5f) * (float)snum / (float)sden - 0.5f) - 1;
    hi = (int)ceilf(((2.f * t + 2.5f) + 0.5f) * (float)snum / (float)sden - 0.5f) + 1;
    if (t == 0) lo = 0;
    if (t == nt - 1) hi = nout - 1;
    lo = max(lo, 0);
    hi = min(hi, nout - 1);
}
// the forward's tap weight of output pixel X (along one axis) on texel t
__device__ __forceinline__ float rhat_weight(int X, int t, int nt, int snum, int sden) {
    const int Q2 = 4 * snum;
    const float inv2Q = 0.25f / (float)snum;
    const int Px = 2 * sden * X + sden - snum;
    const int rx = floor_div(Px - snum, Q2);
    const float fx = (float)(Px - snum - rx * Q2) * inv2Q;
    const int rx0 = clampi(rx, 0, nt - 1), rx1 = clampi(rx + 1, 0, nt - 1);
    return (rx0 == t ? 1.f - fx : 0.f) + (rx1 == t ? fx : 0.f);
}

// the forward's two taps of output pixel X (along one axis): texels rx and rx + 1 (before
// clamping) with weights 1 - fx and fx -- the quantities rhat_weight derives per texel
__device__ __forceinline__ void rhat_taps(int X, int snum, int sden, int &rx, float &fx) {
    const int Q2 = 4 * snum;
    const float inv2Q = 0.25f / (float)snum;
    const int Px = 2 * sden * X + sden - snum;
    rx = floor_div(Px - snum, Q2);
    fx = (float)(Px - snum - rx * Q2) * inv2Q;
}

// the output pixels one block of 128 texel columns reads: at most 4 x 128 + 2 x 13 at 4x
constexpr int kRhatSpan = 1024 + 64;

// R-hat-bar along x: for each output row, texel column u gathers the taps of the output
// pixels in its range.  The block's pixels' taps are derived once into shared memory,
// then every texel sums its own, in pixel order (the sums rhat_weight would give).
__global__ void __launch_bounds__(128) k_rhat_rows(const float *__restrict__ rhbar_pix, Geom g, int snum, int sden,
                                                   int ho, int wo, float *__restrict__ rows) {
    __shared__ int s_rx[kRhatSpan];
    __shared__ float s_fx[kRhatSpan];
    const int u0 = blockIdx.x * blockDim.x, u = u0 + threadIdx.x, Y = blockIdx.y, f = blockIdx.z;
    if (f == g.ref) return;  // the whole block
    int lo0, hi0, lo1, hi1;
    rhat_range(u0, g.wh, wo, snum, sden, lo0, hi0);
    rhat_range(min(u0 + (int)blockDim.x - 1, g.wh - 1), g.wh, wo, snum, sden, lo1, hi1);
    const int xs = lo0, xn = hi1 - lo0 + 1;  // the ranges grow with u: the block reads [lo0, hi1]
    const bool staged = xn <= kRhatSpan;
    if (staged) {
        for (int k = threadIdx.x; k < xn; k += blockDim.x) rhat_taps(xs + k, snum, sden, s_rx[k], s_fx[k]);
    }
    __syncthreads();
    if (u >= g.wh) return;
    int lo, hi;
    rhat_range(u, g.wh, wo, snum, sden, lo, hi);
    const float *row = rhbar_pix + (size_t)f * ho * wo + (size_t)Y * wo;
    float acc = 0.f;
    for (int X = lo; X <= hi; ++X) {
        float w;
        if (staged) {
            const int rx = s_rx[X - xs];
            const float fx = s_fx[X - xs];
            const int rx0 = clampi(rx, 0, g.wh - 1), rx1 = clampi(rx + 1, 0, g.wh - 1);
            w = (rx0 == u ? 1.f - fx : 0.f) + (rx1 == u ? fx : 0.f);
        } else {
            w = rhat_weight(X, u, g.wh, snum, sden);
        }
        if (w != 0.f) acc = fmaf(w, __ldg(row + X), acc);
    }
    rows[((size_t)f * ho + Y) * g.wh + u] = acc;
}

// R-hat-bar along y: the block's texels share their row v, so the weights of the output
// rows in v's range are derived once into shared memory (the values rhat_weight gives)
__global__ void __launch_bounds__(128) k_rhat_cols(const float *__restrict__ rows, Geom g, int snum, int sden,
                                                   int ho, float *__restrict__ rhbar_tex) {
    __shared__ float s_w[kRhatSpan];
    const int u = blockIdx.x * blockDim.x + threadIdx.x, v = blockIdx.y, f = blockIdx.z;
    if (f == g.ref) return;  // the whole block
    int lo, hi;
    rhat_range(v, g.hh, ho, snum, sden, lo, hi);
    const int yn = hi - lo + 1;
    const bool staged = yn <= kRhatSpan;
    if (staged) {
        for (int k = threadIdx.x; k < yn; k += blockDim.x) s_w[k] = rhat_weight(lo + k, v, g.hh, snum, sden);
    }
    __syncthreads();
    if (u >= g.wh) return;
    const float *col = rows + (size_t)f * ho * g.wh + u;
    float acc = 0.f;
    for (int Y = lo; Y <= hi; ++Y) {
        const float w = staged ? s_w[Y - lo] : rhat_weight(Y, v, g.hh, snum, sden);
        if (w != 0.f) acc = fmaf(w, __ldg(col + (size_t)Y * g.wh), acc);
    }
    rhbar_tex[(size_t)f * g.hh * g.wh + (size_t)v * g.wh + u] = acc;
}

constexpr int kRpThreads = 128;

__global__ void __launch_bounds__(kRpThreads) k_rpath(const float *__restrict__ rhbar_tex,
                                                      const unsigned char *__restrict__ flags,
                                                      const float4 *__restrict__ rb, Geom g,
                                                      float2 *__restrict__ vbar_tex, double *__restrict__ partials) {
    __shared__ double s_red[2][kRpThreads];
    const int u = blockIdx.x * blockDim.x + threadIdx.x, v = blockIdx.y, f = blockIdx.z;
    const size_t hw = (size_t)g.hh * g.wh;
    float pt = 0.f, ps = 0.f;
    if (u < g.wh && f != g.ref) {
        // R-bar(u,v) = sum of Rhat-bar over the 5x5 windows whose argmin is (u,v)
        float rbar = 0.f;
        for (int j = -2; j <= 2; ++j)
            for (int i = -2; i <= 2; ++i) {
                const int uu = u + i, vv = v + j;
                if (uu < 0 || uu >= g.wh || vv < 0 || vv >= g.hh) continue;
                const size_t o = (size_t)f * hw + (size_t)vv * g.wh + uu;
                const int bi = flags[o] & 0x1f;
                // window of (uu,vv) picked offset bi = (dj+2)*5 + (di+2): the pixel (uu+di, vv+dj)
                if (uu + (bi % 5 - 2) == u && vv + (bi / 5 - 2) == v) rbar += rhbar_tex[o];
            }
        const size_t o = (size_t)f * hw + (size_t)v * g.wh + u;
        const bool unclamped = (flags[o] & 0x80) != 0;
        const float4 d = rb[o];
        vbar_tex[o] = unclamped ? make_float2(rbar * d.y, rbar * d.z) : make_float2(0.f, 0.f);
        if (unclamped) {
            ps = rbar * d.w;
            pt = -rbar;
        }
    }
    const int tid = threadIdx.x;
    float pv[2] = {ps, pt}, pe[2];
    warp_sums_comp<2>(pv, pe);
    if ((tid & 31) == 0) {
        s_red[0][(tid >> 5) * 2] = (double)pv[0];
        s_red[0][(tid >> 5) * 2 + 1] = (double)pe[0];
        s_red[1][(tid >> 5) * 2] = (double)pv[1];
        s_red[1][(tid >> 5) * 2 + 1] = (double)pe[1];
    }
    __syncthreads();
    if (tid < 2) {
        double acc = 0.0;
        for (int w = 0; w < kRpThreads / 32; ++w) acc += s_red[tid][2 * w] + s_red[tid][2 * w + 1];
        const size_t bid = ((size_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
        partials[bid * 2 + tid] = acc;
    }
}

// ---------------------------------------------------------------------------------------
// deterministic final sums
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ int tile_first(int k, int ntiles, int nout, int snum, int sden, int tile) {
    if (k <= 0) return 0;
    if (k >= ntiles) return nout;
    const int a = k * 2 * snum * tile - sden + snum, b = 2 * sden;
    return min((a + b - 1) / b, nout);
}

constexpr int kRedThreads = 128;

// Neumaier's compensated sum in FP32: s + c carries the exact error of every addition
__device__ __forceinline__ void comp_add(float &s, float &c, float x) {
    const float t = s + x;
    c += (fabsf(s) >= fabsf(x)) ? (s - t) + x : (x - t) + s;
    s = t;
}

// one warp per (frame, tile): the output-pixel and texel contributions of that tile, each
// lane over every 32nd element in a fixed order (compensated FP32: FP64 arithmetic is
// scarce on this GPU), then the lanes in FP64 by a fixed butterfly -- deterministic
__global__ void __launch_bounds__(kRedThreads) k_motion_reduce(const float2 *__restrict__ vbar_pix,
                                                               const float2 *__restrict__ vbar_tex, Geom g, int snum,
                                                               int sden, int ho, int wo, float *__restrict__ grad_motion) {
    const int lane = threadIdx.x & 31;
    const int t = blockIdx.x * (kRedThreads / 32) + (threadIdx.x >> 5);  // (frame, tile) index
    if (t >= g.n * g.ty * g.tx) return;  // the whole warp
    const int f = t / (g.ty * g.tx), r = t - f * g.ty * g.tx, tyi = r / g.tx, txi = r - tyi * g.tx;
    float sx = 0.f, cx = 0.f, sy = 0.f, cy = 0.f;
    if (f != g.ref) {
        const int X0 = tile_first(txi, g.tx, wo, snum, sden, g.tile), X1 = tile_first(txi + 1, g.tx, wo, snum, sden, g.tile);
        const int Y0 = tile_first(tyi, g.ty, ho, snum, sden, g.tile), Y1 = tile_first(tyi + 1, g.ty, ho, snum, sden, g.tile);
        const size_t po = (size_t)ho * wo;
        const float2 *vp = vbar_pix + (size_t)f * po;
        if (X1 - X0 <= 32) {
            // one column per lane: the rows' loads are independent of the sums, so four
            // are in flight at a time
            const bool on = X0 + lane < X1;
            const float2 *cp = vp + (size_t)Y0 * wo + X0 + (on ? lane : 0);
#pragma unroll 4
            for (int Y = Y0; Y < Y1; ++Y, cp += wo) {
                const float2 vb = on ? __ldg(cp) : make_float2(0.f, 0.f);
                comp_add(sx, cx, vb.x);
                comp_add(sy, cy, vb.y);
            }
        } else {
            for (int Y = Y0; Y < Y1; ++Y)
                for (int X = X0 + lane; X < X1; X += 32) {
                    const float2 vb = vp[(size_t)Y * wo + X];
                    comp_add(sx, cx, vb.x);
                    comp_add(sy, cy, vb.y);
                }
        }
        const int ht = g.tile / 2;
        const int u0 = txi * ht, v0 = tyi * ht;
        const int u1 = (txi == g.tx - 1) ? g.wh : min(u0 + ht, g.wh), v1 = (tyi == g.ty - 1) ? g.hh : min(v0 + ht, g.hh);
        const float2 *vt = vbar_tex + (size_t)f * g.hh * g.wh;
        for (int v = v0; v < v1; ++v)
            for (int u = u0 + lane; u < u1; u += 32) {
                const float2 vb = vt[(size_t)v * g.wh + u];
                comp_add(sx, cx, vb.x);
                comp_add(sy, cy, vb.y);
            }
    }
    double dx = (double)sx + (double)cx, dy = (double)sy + (double)cy;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        dx += __shfl_xor_sync(0xffffffffu, dx, o);
        dy += __shfl_xor_sync(0xffffffffu, dy, o);
    }
    if (lane == 0) {
        const size_t o = (((size_t)f * g.ty + tyi) * g.tx + txi) * 2;
        grad_motion[o] = (float)dx;
        grad_motion[o + 1] = (float)dy;
    }
}

__global__ void __launch_bounds__(kRedThreads) k_param_reduce(const double *__restrict__ p6, int n6,
                                                              const double *__restrict__ p2, int n2,
                                                              float *__restrict__ grad_params) {
    __shared__ double s_red[kRedThreads];
    const int q = blockIdx.x, tid = threadIdx.x;  // q = 0..7
    double acc = 0.0;
    if (q < 6)
        for (int k = tid; k < n6; k += kRedThreads) acc += p6[(size_t)k * 6 + q];
    else
        for (int k = tid; k < n2; k += kRedThreads) acc += p2[(size_t)k * 2 + (q - 6)];
    s_red[tid] = acc;
    __syncthreads();
    for (int sstep = kRedThreads / 2; sstep > 0; sstep >>= 1) {
        if (tid < sstep) s_red[tid] += s_red[tid + sstep];
        __syncthreads();
    }
    if (tid == 0) grad_params[q] = (float)s_red[0];
}

}  // namespace

// workspace of the adjoint beyond the forward planes
size_t carve_backward(void *ws, const Geom &g, int ho, int wo, size_t fwd_bytes, BwdPlanes *B) {
    char *base = static_cast<char *>(ws);
    size_t off = fwd_bytes;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off = (off + bytes + 255) & ~(size_t)255;
        return base ? (void *)(base + o) : nullptr;
    };
    const size_t hw = (size_t)g.hh * g.wh, npx = (size_t)ho * wo;
    B->shape = (float4 *)take(sizeof(float4) * g.n * hw);
    B->rb = (float4 *)take(sizeof(float4) * g.n * hw);
    B->flags = (unsigned char *)take(g.n * hw);
    B->rhbar_tex = (float *)take(sizeof(float) * g.n * hw);
    B->vbar_tex = (float2 *)take(sizeof(float2) * g.n * hw);
    B->vbar_pix = (float2 *)take(sizeof(float2) * g.n * npx);
    B->rhbar_pix = (float *)take(sizeof(float) * g.n * npx);
    B->rhbar_rows = (float *)take(sizeof(float) * g.n * (size_t)ho * g.wh);
    B->n_bwd_blocks = div_up(wo, kBwdW) * div_up(ho, kBwdH);
    B->n_rp_blocks = div_up(g.wh, kRpThreads) * g.hh * g.n;
    B->part6 = (double *)take(sizeof(double) * 6 * (size_t)B->n_bwd_blocks);
    B->part2 = (double *)take(sizeof(double) * 2 * (size_t)B->n_rp_blocks);
    B->sel = (unsigned char *)take((size_t)g.n * g.ty * g.tx);
    return off;
}

// The adjoint in four parts (the call orders them; see hmfsr_merge_backward):
//   shape  -- k_shape: the kernel-shape derivatives of every texel (needs the burst only)
//   robust -- k_sel, k_rback, k_argmin: the robustness derivatives (needs the preparation)
//   main   -- k_merge_bwd and the R-hat-bar gather (needs shape and the preparation)
//   finish -- k_rpath and the two reductions (needs robust and main)
cudaError_t launch_bwd_shape(const uint16_t *burst, const Geom &g, const BwdPlanes &B, cudaStream_t s) {
    const dim3 tex_grid(div_up(g.wh, 128), g.hh, g.n);
    k_shape<<<tex_grid, 128, 0, s>>>(burst, g.h, g.pitch, g.hh, g.wh, g.wl, B.shape);
    return cudaGetLastError();
}

cudaError_t launch_bwd_robust(const float *motion, const Geom &g, const MergeConsts &c, const MergePlanes &P,
                              const BwdPlanes &B, cudaStream_t s) {
    const float2 *mv = reinterpret_cast<const float2 *>(motion);
    const dim3 tex_grid(div_up(g.wh, 128), g.hh, g.n);
    k_sel<<<div_up(g.n * g.ty * g.tx, 128), 128, 0, s>>>(mv, g.n, g.ty, g.tx, c.m_th, B.sel);
    k_rback<<<tex_grid, 128, 0, s>>>(P.s1, P.base_stats, mv, P.s_tile, B.sel, g, c, B.rb, B.flags);
    k_argmin<<<tex_grid, 128, 0, s>>>(B.rb, g, B.flags);
    return cudaGetLastError();
}

cudaError_t launch_bwd_main(const uint16_t *burst, const float *motion, const Geom &g, const MergeConsts &c,
                            const MergePlanes &P, const BwdPlanes &B, int snum, int sden, const float *rgb,
                            const float *lden, const float *grad_rgb, cudaStream_t s) {
    const int ho = (int)(((long long)g.h * snum) / sden), wo = (int)(((long long)g.w * snum) / sden);
    const float2 *mv = reinterpret_cast<const float2 *>(motion);
    const dim3 tex_grid(div_up(g.wh, 128), g.hh, g.n);
    k_merge_bwd<<<dim3(div_up(wo, kBwdW), div_up(ho, kBwdH)), dim3(kBwdW, kBwdH), 0, s>>>(
        burst, mv, g, c, P.kern, B.shape, P.rhat, snum, sden, ho, wo, rgb, lden, grad_rgb, B.vbar_pix, B.rhbar_pix,
        B.part6);
    k_rhat_rows<<<dim3(div_up(g.wh, 128), ho, g.n), 128, 0, s>>>(B.rhbar_pix, g, snum, sden, ho, wo, B.rhbar_rows);
    k_rhat_cols<<<tex_grid, 128, 0, s>>>(B.rhbar_rows, g, snum, sden, ho, B.rhbar_tex);
    return cudaGetLastError();
}

cudaError_t launch_bwd_finish(const Geom &g, const BwdPlanes &B, int snum, int sden, float *grad_params,
                              float *grad_motion, cudaStream_t s) {
    const int ho = (int)(((long long)g.h * snum) / sden), wo = (int)(((long long)g.w * snum) / sden);
    k_rpath<<<dim3(div_up(g.wh, kRpThreads), g.hh, g.n), kRpThreads, 0, s>>>(B.rhbar_tex, B.flags, B.rb, g,
                                                                           B.vbar_tex, B.part2);
    k_motion_reduce<<<div_up(g.n * g.ty * g.tx, kRedThreads / 32), kRedThreads, 0, s>>>(B.vbar_pix, B.vbar_tex, g, snum,
                                                                                      sden, ho, wo, grad_motion);
    k_param_reduce<<<8, kRedThreads, 0, s>>>(B.part6, B.n_bwd_blocks, B.part2, B.n_rp_blocks, grad_params);
    return cudaGetLastError();
}

}  // namespace hmfsr
