// The accumulation (Eq. 1-2): per output pixel, every frame's 3x3 Bayer window
// weighted by the anisotropic kernel and the robustness, with a fused normalisation.
// Shared by the per-burst kernel and the batched persistent kernel.
#pragma once

#include "stages.cuh"

namespace hmfsr {
namespace stage {

// ======================================================================================
// accumulation (Eq. 1-2)
// ======================================================================================
// --------------------------------------------------------------------------------------
// accumulation (Eq. 1-2): one thread per output pixel, all frames, registers only
// --------------------------------------------------------------------------------------
constexpr int kMergeW = 32, kMergeH = 4;


// The 3x3 Bayer neighbourhood of frame sample rows around (kx, ky): raw values and the
// weight exponents q' (log2 units) of the quadratic form; samples outside the frame get
// q' = +inf.  kBorder selects the checked variant.
template <bool kBorder>
__device__ __forceinline__ void gather3x3(const uint16_t *__restrict__ fr, int pitch, int h, int w, int kx, int ky,
                                          const float (&Ax)[3], const float (&Ex)[3], const float (&Cy)[3],
                                          const float (&dys)[3], float (&q)[3][3], float (&rv)[3][3]) {
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        const int yy = ky - 1 + j;
        const bool yok = !kBorder || ((unsigned)yy < (unsigned)h);
        const int row = (kBorder ? clampi(yy, 0, h - 1) : yy) * pitch;  // 32-bit: frames hold < 2^31 samples
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            const int xx = kx - 1 + i;
            rv[j][i] = (float)__ldg(fr + row + (kBorder ? clampi(xx, 0, w - 1) : xx));
            const float qq = fmaf(Ex[i], dys[j], Ax[i] + Cy[j]);
            if (kBorder) q[j][i] = (yok && (unsigned)xx < (unsigned)w) ? qq : INFINITY;
            else q[j][i] = qq;
        }
    }
}

// running sums of one output pixel: Eq. 1's numerator and denominator per channel, each
// scaled by 2^-m with a per-channel exponent shift m (log2 units)
struct PixelAcc {
    float numR = 0.f, numG = 0.f, numB = 0.f, denR = 0.f, denG = 0.f, denB = 0.f;
    float mR = kBig, mG = kBig, mB = kBig;
};

// One frame's contribution (Eq. 1-2) to one pixel from the weight exponents q' and
// values of its 3x3 window; cg: the window's centre sample is green; sw: its centre row
// is odd (the Bayer arrangement of the window).
__device__ __forceinline__ void accumulate_frame(const float (&q)[3][3], const float (&rv)[3][3], float rh, bool cg,
                                                 bool sw, PixelAcc &a) {
    // per-class minima: C = centre, H = (+-1, 0), V = (0, +-1), K = corners
    const float qC = q[1][1];
    const float mH = fminf(q[1][0], q[1][2]), mV = fminf(q[0][1], q[2][1]);
    const float mK = fminf(fminf(q[0][0], q[0][2]), fminf(q[2][0], q[2][2]));
    const float f1 = cg ? mH : qC, f2 = cg ? mV : mK, fG = cg ? fminf(qC, mK) : fminf(mH, mV);
    const float fR = sw ? f2 : f1, fB = sw ? f1 : f2;
    if (fR < a.mR - 64.f || fG < a.mG - 64.f || fB < a.mB - 64.f) {
        // move a channel's shift down to this frame's minimum (rare after the base frame)
        if (fR < a.mR - 64.f) { const float s = fast_exp2(fR - a.mR); a.numR *= s; a.denR *= s; a.mR = fR; }
        if (fG < a.mG - 64.f) { const float s = fast_exp2(fG - a.mG); a.numG *= s; a.denG *= s; a.mG = fG; }
        if (fB < a.mB - 64.f) { const float s = fast_exp2(fB - a.mB); a.numB *= s; a.denB *= s; a.mB = fB; }
    }
    const float mS1 = sw ? a.mB : a.mR, mS2 = sw ? a.mR : a.mB;
    const float sC = cg ? a.mG : mS1, sK = cg ? a.mG : mS2, sH = cg ? mS1 : a.mG, sV = cg ? mS2 : a.mG;
    float w;
    w = fast_exp2(sC - q[1][1]);
    const float nC = w * rv[1][1], dC = w;
    w = fast_exp2(sH - q[1][0]);
    float nH = w * rv[1][0], dH = w;
    w = fast_exp2(sH - q[1][2]);
    nH = fmaf(w, rv[1][2], nH); dH += w;
    w = fast_exp2(sV - q[0][1]);
    float nV = w * rv[0][1], dV = w;
    w = fast_exp2(sV - q[2][1]);
    nV = fmaf(w, rv[2][1], nV); dV += w;
    w = fast_exp2(sK - q[0][0]);
    float nK = w * rv[0][0], dK = w;
    w = fast_exp2(sK - q[0][2]);
    nK = fmaf(w, rv[0][2], nK); dK += w;
    w = fast_exp2(sK - q[2][0]);
    nK = fmaf(w, rv[2][0], nK); dK += w;
    w = fast_exp2(sK - q[2][2]);
    nK = fmaf(w, rv[2][2], nK); dK += w;
    const float n1 = cg ? nH : nC, n2 = cg ? nV : nK, nG = cg ? nC + nK : nH + nV;
    const float d1 = cg ? dH : dC, d2 = cg ? dV : dK, dG = cg ? dC + dK : dH + dV;
    a.numR = fmaf(rh, sw ? n2 : n1, a.numR);
    a.denR = fmaf(rh, sw ? d2 : d1, a.denR);
    a.numB = fmaf(rh, sw ? n1 : n2, a.numB);
    a.denB = fmaf(rh, sw ? d1 : d2, a.denB);
    a.numG = fmaf(rh, nG, a.numG);
    a.denG = fmaf(rh, dG, a.denG);
}

// floor(a / B) for B > 0: an arithmetic shift when B is a compile-time power of two,
// the exact integer floor division otherwise (B = 0: use the runtime divisor b)
template <int B>
__device__ __forceinline__ int floor_div_q(int a, int b) {
    if constexpr (B > 0 && (B & (B - 1)) == 0) {
        int sh = 0;
        while ((1 << sh) < B) ++sh;
        return a >> sh;
    } else if constexpr (B > 0) {
        return floor_div(a, B);
    } else {
        return floor_div(a, b);
    }
}

// Window geometry of one motion tile of one frame for Q = 2 x (output px per raw px
// numerator): {floor(Q vx), floor(Q vy)} exactly and the fractions {Q vx - F, Q vy - F}
// (Sec. 5.1: the window centre and the kernel's sampling point).  The base frame's entry
// is zero: its motion is zero by definition.  i runs over n x tiles.
__device__ __forceinline__ void geo_entry(const float2 *__restrict__ motion, int n, int ntl, int ref, int Q,
                                          int4 *__restrict__ geo, int i) {
    if (i >= n * ntl) return;
    int4 e = make_int4(0, 0, 0, 0);
    if (i / ntl != ref) {
        const float2 mv = motion[i];
        const int FX = floor_mul(Q, mv.x), FY = floor_mul(Q, mv.y);
        const float fQ = (float)Q;
        e = make_int4(FX, FY, __float_as_int(fmaf(fQ, mv.x, -(float)FX)), __float_as_int(fmaf(fQ, mv.y, -(float)FY)));
    }
    geo[i] = e;
}

// SN/SD > 0: compile-time output scale SN/SD (constant divisors); 0: runtime snum/sden.
// geo: the window geometry of every (frame, motion tile) for this scale (geo_entry).
template <bool kDen, int SN, int SD>
__device__ __forceinline__ void merge_px(const uint16_t *__restrict__ burst, const int4 *__restrict__ geo,
                                         const Geom &g, const float4 *__restrict__ kern,
                                         const float *__restrict__ rhat_planes, int snum_rt, int sden_rt, int ho, int wo,
                                         float *__restrict__ rgb, float *__restrict__ den_out, int X, int Y) {
    if (X < 0 || Y < 0 || X >= wo || Y >= ho) return;
    constexpr int QC = 2 * SN, Q2C = 4 * SN;
    const int snum = SN > 0 ? SN : snum_rt, sden = SD > 0 ? SD : sden_rt;
    const int Q = 2 * snum, Q2 = 4 * snum;
    const float fQ = (float)Q, invQ = 1.f / fQ, inv2Q = 0.5f / fQ;
    // output pixel centre x0 = Px / Q in raw px (exact rational)
    const int Px = 2 * sden * X + sden - snum, Py = 2 * sden * Y + sden - snum;
    const int txi = min(max(floor_div(Px, Q * g.tile), 0), g.tx - 1);
    const int tyi = min(max(floor_div(Py, Q * g.tile), 0), g.ty - 1);
    const size_t hw = (size_t)g.hh * g.wh, ntl = (size_t)g.ty * g.tx;
    const int4 *geo_px = geo + (size_t)tyi * g.tx + txi;
    // Rhat is sampled on the base half-res grid at (x0 - 1/2)/2 = (P - num) / 2Q
    const int rx = floor_div_q<Q2C>(Px - snum, Q2), ry = floor_div_q<Q2C>(Py - snum, Q2);
    const float rfx = (float)(Px - snum - rx * Q2) * inv2Q, rfy = (float)(Py - snum - ry * Q2) * inv2Q;
    const int rx0 = clampi(rx, 0, g.wh - 1), rx1 = clampi(rx + 1, 0, g.wh - 1);
    const int ry0 = clampi(ry, 0, g.hh - 1), ry1 = clampi(ry + 1, 0, g.hh - 1);
    const int r00 = ry0 * g.wh + rx0, r10 = ry0 * g.wh + rx1, r01 = ry1 * g.wh + rx0, r11 = ry1 * g.wh + rx1;
    const float rw00 = (1.f - rfx) * (1.f - rfy), rw10 = rfx * (1.f - rfy), rw01 = (1.f - rfx) * rfy, rw11 = rfx * rfy;
    // a frame's robustness at this pixel (1 for the base frame)
    auto rhat_at = [&](int f) -> float {
        if (f == g.ref) return 1.f;
        const float *Rp = rhat_planes + (size_t)f * hw;
        return fmaf(rw00, __ldg(Rp + r00), fmaf(rw10, __ldg(Rp + r10), fmaf(rw01, __ldg(Rp + r01), rw11 * __ldg(Rp + r11))));
    };

    PixelAcc acc;
    const size_t fstride = (size_t)g.h * g.pitch;

    // frames in the order base frame, then the others; the next frame's geometry and
    // robustness are fetched while this one is merged
    int f_nx = g.ref;
    int4 geo_nx = __ldg(geo_px + (size_t)f_nx * ntl);
    float rh_nx = 1.f;
    for (int it = 0; it < g.n; ++it) {
        const int f = f_nx;
        const int4 gq = geo_nx;
        const float rh = rh_nx;
        if (it + 1 < g.n) {
            f_nx = (it + 1 <= g.ref) ? it : it + 1;
            geo_nx = __ldg(geo_px + (size_t)f_nx * ntl);
            rh_nx = rhat_at(f_nx);
        }
        if (!(rh > 0.f)) continue;  // a rejected frame adds nothing
        // window centre k = round(x0 + v) (ties up), exactly: F = floor(Q v)
        const int FX = gq.x, FY = gq.y;
        const float zx = __int_as_float(gq.z), zy = __int_as_float(gq.w);  // Q v - F
        const int kx = floor_div_q<QC>(Px + snum + FX, Q), ky = floor_div_q<QC>(Py + snum + FY, Q);
        // offset of the centre sample from x0 + v: (kx Q - Px - F - (Q v - F)) / Q
        const float dx0 = ((float)(kx * Q - Px - FX) - zx) * invQ;
        const float dy0 = ((float)(ky * Q - Py - FY) - zy) * invQ;
        // Omega is sampled on frame f's half-res grid at (x0 + v - 1/2)/2
        const int gx = Px - snum + FX, gy = Py - snum + FY;
        const int ox = floor_div_q<Q2C>(gx, Q2), oy = floor_div_q<Q2C>(gy, Q2);
        const float ofx = ((float)(gx - ox * Q2) + zx) * inv2Q, ofy = ((float)(gy - oy * Q2) + zy) * inv2Q;
        const int ox0 = clampi(ox, 0, g.wh - 1), ox1 = clampi(ox + 1, 0, g.wh - 1);
        const int oy0 = clampi(oy, 0, g.hh - 1) * g.wh, oy1 = clampi(oy + 1, 0, g.hh - 1) * g.wh;
        const float4 *K = kern + (size_t)f * hw;
        const float4 t0 = __ldg(K + (oy0 + ox0)), t1 = __ldg(K + (oy0 + ox1));
        const float4 t2 = __ldg(K + (oy1 + ox0)), t3 = __ldg(K + (oy1 + ox1));
        const float b0 = (1.f - ofx) * (1.f - ofy), b1 = ofx * (1.f - ofy), b2 = (1.f - ofx) * ofy, b3 = ofx * ofy;
        // Omega = a I + M, M = sum_k g_k u_k u_k^T;  adj(Omega) = a I + sum_k g_k u_k^perp u_k^perp^T
        // (the library is built without automatic FMA contraction; the fused
        // multiply-adds below are written out so the arithmetic is the same wherever this
        // function is inlined)
        const float a = fmaf(b0, t0.x, fmaf(b1, t1.x, fmaf(b2, t2.x, b3 * t3.x)));
        const float g0 = b0 * t0.y, g1 = b1 * t1.y, g2 = b2 * t2.y, g3 = b3 * t3.y;
        const float gw0 = g0 * t0.w, gw1 = g1 * t1.w, gw2 = g2 * t2.w, gw3 = g3 * t3.w;
        const float gz0 = g0 * t0.z, gz1 = g1 * t1.z, gz2 = g2 * t2.z, gz3 = g3 * t3.z;
        const float Nxx = fmaf(gw0, t0.w, fmaf(gw1, t1.w, fmaf(gw2, t2.w, gw3 * t3.w)));
        const float Nyy = fmaf(gz0, t0.z, fmaf(gz1, t1.z, fmaf(gz2, t2.z, gz3 * t3.z)));
        const float Nxy = -fmaf(gw0, t0.z, fmaf(gw1, t1.z, fmaf(gw2, t2.z, gw3 * t3.z)));
        const float Gs = (g0 + g1) + (g2 + g3);
        // det(M) = sum_{k<l} g_k g_l (u_k x u_l)^2 (Cauchy-Binet: all terms >= 0)
        const float c01 = fmaf(t0.z, t1.w, -(t0.w * t1.z)), c02 = fmaf(t0.z, t2.w, -(t0.w * t2.z));
        const float c03 = fmaf(t0.z, t3.w, -(t0.w * t3.z)), c12 = fmaf(t1.z, t2.w, -(t1.w * t2.z));
        const float c13 = fmaf(t1.z, t3.w, -(t1.w * t3.z)), c23 = fmaf(t2.z, t3.w, -(t2.w * t3.z));
        const float s0 = fmaf(g1 * c01, c01, fmaf(g2 * c02, c02, (g3 * c03) * c03));
        const float s1 = fmaf(g2 * c12, c12, (g3 * c13) * c13);
        const float detM = fmaf(g0, s0, fmaf(g1, s1, (g2 * g3) * (c23 * c23)));
        const float det = fmaf(a, a + Gs, detM);
        const float sc = kHalfLog2e * fast_rcp(det);
        // q'(d) = (d^T adj(Omega) d) / det * log2(e)/2: weight = 2^-q'
        const float Bxx = (a + Nxx) * sc, Byy = (a + Nyy) * sc, Bxy2 = 2.f * Nxy * sc;
        const float dxs[3] = {dx0 - 1.f, dx0, dx0 + 1.f};
        const float dys[3] = {dy0 - 1.f, dy0, dy0 + 1.f};
        float Ax[3], Ex[3], Cy[3];
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            Ax[i] = Bxx * dxs[i] * dxs[i];
            Ex[i] = Bxy2 * dxs[i];
            Cy[i] = Byy * dys[i] * dys[i];
        }
        // the 3x3 Bayer neighbourhood; samples outside the frame are left out
        const uint16_t *fr = burst + (size_t)f * fstride;
        float q[3][3], rv[3][3];
        if ((unsigned)(kx - 1) < (unsigned)(g.w - 2) && (unsigned)(ky - 1) < (unsigned)(g.h - 2))
            gather3x3<false>(fr, g.pitch, g.h, g.w, kx, ky, Ax, Ex, Cy, dys, q, rv);
        else
            gather3x3<true>(fr, g.pitch, g.h, g.w, kx, ky, Ax, Ex, Cy, dys, q, rv);
        // Bayer arrangement of the window: cg = centre sample is green; sw = centre row is odd
        accumulate_frame(q, rv, rh, ((kx ^ ky) & 1) != 0, (ky & 1) != 0, acc);
    }
    const size_t po = (size_t)ho * wo, o = (size_t)Y * wo + X;
    rgb[o] = acc.numR / acc.denR;
    rgb[po + o] = acc.numG / acc.denG;
    rgb[2 * po + o] = acc.numB / acc.denB;
    if (kDen) {
        den_out[o] = log2f(acc.denR) - acc.mR;
        den_out[po + o] = log2f(acc.denG) - acc.mG;
        den_out[2 * po + o] = log2f(acc.denB) - acc.mB;
    }
}

}  // namespace stage
}  // namespace hmfsr
