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
            rv[j][i] = (float)HMFSR_LDG(fr + row + (kBorder ? clampi(xx, 0, w - 1) : xx));
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

// The same contribution from the quadratic form's parts instead of its values: per
// window column i, A[i] = Bxx dx_i^2 and E[i] = Bxy2 dx_i; per row j, C[j] = Byy dy_j^2
// and dy[j]; q' = A[i] + C[j] + E[i] dy[j].  Each sample's weight is taken directly as
// 2^t with t = m - q', m the exponent shift of its channel, folded into per-row terms
// (m - C[j]) so that no sample needs its channel's shift selected.  While every t stays
// at or below 64 no channel's shift has to move; otherwise (the first frame, whose
// shifts start at +inf, and the rare frame that brings a sample far closer) the frame
// takes accumulate_frame, which moves the shifts.  kBorder: `ok` marks the samples
// inside the frame (the others are left out).
template <bool kBorder>
__device__ __forceinline__ void accumulate_frame_parts(const float (&A)[3], const float (&E)[3], const float (&C)[3],
                                                       const float (&dy)[3], const float (&rv)[3][3],
                                                       const bool (&ok)[3][3], float rh, bool cg, bool sw,
                                                       PixelAcc &a) {
    // the shifts of the four sample classes: C = centre, H = (+-1, 0), V = (0, +-1), K = corners
    const float mS1 = sw ? a.mB : a.mR, mS2 = sw ? a.mR : a.mB;
    const float sC = cg ? a.mG : mS1, sK = cg ? a.mG : mS2, sH = cg ? mS1 : a.mG, sV = cg ? mS2 : a.mG;
    const float rowK0 = sK - C[0], rowV0 = sV - C[0], rowH1 = sH - C[1], rowC1 = sC - C[1];
    const float rowK2 = sK - C[2], rowV2 = sV - C[2];
    float t[3][3];
    t[0][0] = fmaf(-E[0], dy[0], rowK0 - A[0]);
    t[0][1] = fmaf(-E[1], dy[0], rowV0 - A[1]);
    t[0][2] = fmaf(-E[2], dy[0], rowK0 - A[2]);
    t[1][0] = fmaf(-E[0], dy[1], rowH1 - A[0]);
    t[1][1] = fmaf(-E[1], dy[1], rowC1 - A[1]);
    t[1][2] = fmaf(-E[2], dy[1], rowH1 - A[2]);
    t[2][0] = fmaf(-E[0], dy[2], rowK2 - A[0]);
    t[2][1] = fmaf(-E[1], dy[2], rowV2 - A[1]);
    t[2][2] = fmaf(-E[2], dy[2], rowK2 - A[2]);
    float tmax = -INFINITY;
#pragma unroll
    for (int j = 0; j < 3; ++j)
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            if (kBorder && !ok[j][i]) t[j][i] = -INFINITY;
            tmax = fmaxf(tmax, t[j][i]);
        }
    if (!(tmax <= 64.f)) {
        // a shift has to move (or every sample is outside the frame): the exponents q'
        float q[3][3];
#pragma unroll
        for (int j = 0; j < 3; ++j)
#pragma unroll
            for (int i = 0; i < 3; ++i)
                q[j][i] = (kBorder && !ok[j][i]) ? INFINITY : fmaf(E[i], dy[j], A[i] + C[j]);
        accumulate_frame(q, rv, rh, cg, sw, a);
        return;
    }
    float w;
    w = fast_exp2(t[1][1]);
    const float nC = w * rv[1][1], dC = w;
    w = fast_exp2(t[1][0]);
    float nH = w * rv[1][0], dH = w;
    w = fast_exp2(t[1][2]);
    nH = fmaf(w, rv[1][2], nH); dH += w;
    w = fast_exp2(t[0][1]);
    float nV = w * rv[0][1], dV = w;
    w = fast_exp2(t[2][1]);
    nV = fmaf(w, rv[2][1], nV); dV += w;
    w = fast_exp2(t[0][0]);
    float nK = w * rv[0][0], dK = w;
    w = fast_exp2(t[0][2]);
    nK = fmaf(w, rv[0][2], nK); dK += w;
    w = fast_exp2(t[2][0]);
    nK = fmaf(w, rv[2][0], nK); dK += w;
    w = fast_exp2(t[2][2]);
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
        const float2 mv = HMFSR_LD(motion + i);
        const int FX = floor_mul(Q, mv.x), FY = floor_mul(Q, mv.y);
        const float fQ = (float)Q;
        e = make_int4(FX, FY, __float_as_int(fmaf(fQ, mv.x, -(float)FX)), __float_as_int(fmaf(fQ, mv.y, -(float)FY)));
    }
    HMFSR_ST(geo + i, e);
}

// The quadratic form of Eq. 2 for Omega interpolated bilinearly (weights b0..b3) from
// four texels t = {a, delta, ux, uy} (Omega = a I + delta u u^T): q'(d) = (d^T adj(Omega) d)
// / det(Omega) x log2(e)/2 = Bxx dx^2 + Bxy2 dx dy + Byy dy^2, so that a sample's weight
// is 2^-q'.  Omega = a I + M with M = sum_k g_k u_k u_k^T, g_k = b_k delta_k >= 0, and
// adj(Omega) = a I + sum_k g_k u_k^perp u_k^perp^T.  det(Omega) = a^2 + a sum_k g_k +
// det(M), with det(M) = sum_{k<l} g_k g_l (u_k x u_l)^2 (Cauchy-Binet): every term >= 0,
// so nothing cancels however elongated the kernels are.  (The library is built without
// automatic FMA contraction; the fused multiply-adds are written out, so the arithmetic
// is the same wherever this is inlined.)
__device__ __forceinline__ void omega_form(const float4 &t0, const float4 &t1, const float4 &t2, const float4 &t3,
                                           float b0, float b1, float b2, float b3, float &Bxx, float &Byy,
                                           float &Bxy2) {
    const float a = fmaf(b0, t0.x, fmaf(b1, t1.x, fmaf(b2, t2.x, b3 * t3.x)));
    const float g0 = b0 * t0.y, g1 = b1 * t1.y, g2 = b2 * t2.y, g3 = b3 * t3.y;
    const float gw0 = g0 * t0.w, gw1 = g1 * t1.w, gw2 = g2 * t2.w, gw3 = g3 * t3.w;
    const float gz0 = g0 * t0.z, gz1 = g1 * t1.z, gz2 = g2 * t2.z, gz3 = g3 * t3.z;
    const float Nxx = fmaf(gw0, t0.w, fmaf(gw1, t1.w, fmaf(gw2, t2.w, gw3 * t3.w)));
    const float Nyy = fmaf(gz0, t0.z, fmaf(gz1, t1.z, fmaf(gz2, t2.z, gz3 * t3.z)));
    const float Nxy = -fmaf(gw0, t0.z, fmaf(gw1, t1.z, fmaf(gw2, t2.z, gw3 * t3.z)));
    const float Gs = (g0 + g1) + (g2 + g3);
    const float c01 = fmaf(t0.z, t1.w, -(t0.w * t1.z)), c02 = fmaf(t0.z, t2.w, -(t0.w * t2.z));
    const float c03 = fmaf(t0.z, t3.w, -(t0.w * t3.z)), c12 = fmaf(t1.z, t2.w, -(t1.w * t2.z));
    const float c13 = fmaf(t1.z, t3.w, -(t1.w * t3.z)), c23 = fmaf(t2.z, t3.w, -(t2.w * t3.z));
    const float s0 = fmaf(g1 * c01, c01, fmaf(g2 * c02, c02, (g3 * c03) * c03));
    const float s1 = fmaf(g2 * c12, c12, (g3 * c13) * c13);
    const float detM = fmaf(g0, s0, fmaf(g1, s1, (g2 * g3) * (c23 * c23)));
    const float det = fmaf(a, a + Gs, detM);
    const float sc = kHalfLog2e * fast_rcp(det);
    Bxx = (a + Nxx) * sc;
    Byy = (a + Nyy) * sc;
    Bxy2 = 2.f * Nxy * sc;
}

// The accumulation in chunks of frames (bounded memory): the running sums of every output
// pixel travel between launches in a state buffer of 9 planes of Ho x Wo floats
// {numR, numG, numB, denR, denG, denB, mR, mG, mB}.  state_in: the sums so far (nullptr
// for the first chunk, which starts empty); state_out: where to leave them (nullptr for
// the last chunk, which normalises into the RGB output instead); skip_base: this chunk's
// burst holds the base frame only for the robustness statistics, and its contribution was
// made by an earlier chunk.  A pixel's state is read and written by the thread that owns
// it, so state_in may equal state_out.
struct ChunkIO {
    const float *state_in = nullptr;
    float *state_out = nullptr;
    int skip_base = 0;
    size_t plane = 0;  // Ho x Wo
};

__device__ __forceinline__ void load_state(const ChunkIO &io, size_t o, PixelAcc &a) {
    const float *p = io.state_in + o;
    const size_t q = io.plane;
    a.numR = HMFSR_LD(p); a.numG = HMFSR_LD(p + q); a.numB = HMFSR_LD(p + 2 * q);
    a.denR = HMFSR_LD(p + 3 * q); a.denG = HMFSR_LD(p + 4 * q); a.denB = HMFSR_LD(p + 5 * q);
    a.mR = HMFSR_LD(p + 6 * q); a.mG = HMFSR_LD(p + 7 * q); a.mB = HMFSR_LD(p + 8 * q);
}

__device__ __forceinline__ void store_state(const ChunkIO &io, size_t o, const PixelAcc &a) {
    float *p = io.state_out + o;
    const size_t q = io.plane;
    HMFSR_ST(p, a.numR); HMFSR_ST(p + q, a.numG); HMFSR_ST(p + 2 * q, a.numB);
    HMFSR_ST(p + 3 * q, a.denR); HMFSR_ST(p + 4 * q, a.denG); HMFSR_ST(p + 5 * q, a.denB);
    HMFSR_ST(p + 6 * q, a.mR); HMFSR_ST(p + 7 * q, a.mG); HMFSR_ST(p + 8 * q, a.mB);
}

// frame of step `it` of the accumulation order: the base frame, then the others in order
__device__ __forceinline__ int frame_of_step(int it, int ref) { return it == 0 ? ref : (it <= ref ? it - 1 : it); }

// SN/SD > 0: compile-time output scale SN/SD (constant divisors); 0: runtime snum/sden.
// geo: the window geometry of every (frame, motion tile) for this scale (geo_entry).
template <bool kDen, int SN, int SD, bool kChunk = false>
__device__ __forceinline__ void merge_px(const uint16_t *__restrict__ burst, const int4 *__restrict__ geo,
                                         const Geom &g, const float4 *__restrict__ kern,
                                         const float *__restrict__ rhat_planes, int snum_rt, int sden_rt, int ho, int wo,
                                         float *__restrict__ rgb, float *__restrict__ den_out, int X, int Y,
                                         const ChunkIO &io = ChunkIO{}) {
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
        return fmaf(rw00, HMFSR_LDG(Rp + r00), fmaf(rw10, HMFSR_LDG(Rp + r10), fmaf(rw01, HMFSR_LDG(Rp + r01), rw11 * HMFSR_LDG(Rp + r11))));
    };

    PixelAcc acc;
    const size_t fstride = (size_t)g.h * g.pitch;
    int it0 = 0;
    if constexpr (kChunk) {
        if (io.state_in) load_state(io, (size_t)Y * wo + X, acc);
        it0 = io.skip_base ? 1 : 0;
    }

    // frames in the order base frame, then the others; each frame's geometry and
    // robustness are read at the top of its own iteration (fetching them a frame ahead
    // spilled at 1.5x and measured 1.5-3% slower)
    int f_nx = kChunk ? frame_of_step(it0, g.ref) : g.ref;
    for (int it = it0; it < g.n; ++it) {
        const int f = f_nx;
        const int4 gq = HMFSR_LDG(geo_px + (size_t)f * ntl);
        const float rh = rhat_at(f);
        if (it + 1 < g.n) f_nx = (it + 1 <= g.ref) ? it : it + 1;
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
        const float4 t0 = HMFSR_LDG(K + (oy0 + ox0)), t1 = HMFSR_LDG(K + (oy0 + ox1));
        const float4 t2 = HMFSR_LDG(K + (oy1 + ox0)), t3 = HMFSR_LDG(K + (oy1 + ox1));
        const float b0 = (1.f - ofx) * (1.f - ofy), b1 = ofx * (1.f - ofy), b2 = (1.f - ofx) * ofy, b3 = ofx * ofy;
        float Bxx, Byy, Bxy2;
        omega_form(t0, t1, t2, t3, b0, b1, b2, b3, Bxx, Byy, Bxy2);
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
    if constexpr (kChunk) {
        if (io.state_out) {
            store_state(io, o, acc);
            return;
        }
    }
    HMFSR_ST(rgb + o, acc.numR / acc.denR);
    HMFSR_ST(rgb + po + o, acc.numG / acc.denG);
    HMFSR_ST(rgb + 2 * po + o, acc.numB / acc.denB);
    if (kDen) {
        HMFSR_ST(den_out + o, log2f(acc.denR) - acc.mR);
        HMFSR_ST(den_out + po + o, log2f(acc.denG) - acc.mG);
        HMFSR_ST(den_out + 2 * po + o, log2f(acc.denB) - acc.mB);
    }
}


// ======================================================================================
// accumulation at scale 1 (Eq. 1-2): one thread per 2 x NY block of output pixels
// ======================================================================================
// At scale 1 output pixel X sits at raw x0 = X and the motion tile is chosen by the base
// position, so the pixels of an even-aligned 2 x NY block lie in one tile and share the
// frame's motion v.  Their window centres are (kx, ky) + (pa, pb) with kx = X + round(vx),
// so their 3x3 windows together are one 4 x (NY + 2) raw block: 16 loads instead of 36
// for a 2 x 2 block.  The offsets of the samples from x0 + v are the same for every pixel
// (they depend on round(v) - v only), so the squares dx^2 and dy^2 of Eq. 2 are formed
// once per block and frame.  Each pixel interpolates Omega at its own position on frame
// f's half-res grid and Rhat at its own position on the base grid, and takes its window's
// Bayer arrangement from the parity of its centre (accumulate_frame).
constexpr int kQuadW = 32;  // output pixels per block row: 4 warps of 8 x 4 threads, 2 x 2 warps
// output rows per thread: 2 (2 x 2 pixels, 128 registers, 4 blocks per SM) measured
// faster than 1 (2 x 1 pixels, 96 registers) at 12 MP x 8: 1.15 against 1.27 ms
constexpr int kQuadNY = 2;

// Where the Omega texels of a frame come from for a pixel of the block: plane K (wh x hh
// texels), the block's texel column u and the texel row of its first pixel row, and per
// pixel column (pa) / row (pb) the cell offset and the fraction.
template <int NY>
struct QuadOmega {
    const float4 *K;
    int wh, hh, u, v;
    int Ox[2], Oy[NY];
    float fx[2], fy[NY];
};

// Omega's quadratic form for pixel (pa, pb) of the block: the texel cell with top-left
// (u + Ox[pa], v + Oy[pb]) at fractions (fx[pa], fy[pb]); kBorder clamps the texel
// indices to the plane.
template <bool kBorder, int NY>
__device__ __forceinline__ void quad_omega(const QuadOmega<NY> &om, int pa, int pb, float &Bxx, float &Byy,
                                           float &Bxy2) {
    int c0 = om.u + om.Ox[pa], c1 = c0 + 1, r0 = om.v + om.Oy[pb], r1 = r0 + 1;
    if (kBorder) {
        c0 = clampi(c0, 0, om.wh - 1);
        c1 = clampi(c1, 0, om.wh - 1);
        r0 = clampi(r0, 0, om.hh - 1);
        r1 = clampi(r1, 0, om.hh - 1);
    }
    const float4 *R0 = om.K + (size_t)r0 * om.wh, *R1 = om.K + (size_t)r1 * om.wh;
    const float4 t0 = HMFSR_LDG(R0 + c0), t1 = HMFSR_LDG(R0 + c1), t2 = HMFSR_LDG(R1 + c0), t3 = HMFSR_LDG(R1 + c1);
    const float ofx = om.fx[pa], ofy = om.fy[pb];
    const float b0 = (1.f - ofx) * (1.f - ofy), b1 = ofx * (1.f - ofy), b2 = (1.f - ofx) * ofy, b3 = ofx * ofy;
    omega_form(t0, t1, t2, t3, b0, b1, b2, b3, Bxx, Byy, Bxy2);
}

// The 4 x (NY + 2) raw block with first sample (bx, by) of frame fr; kBorder clamps reads
// to the frame and reports which columns and rows lie inside it.
template <bool kBorder, int NY>
__device__ __forceinline__ void quad_block(const uint16_t *__restrict__ fr, int pitch, int h, int w, int bx, int by,
                                           float (&rv)[NY + 2][4], bool (&cok)[4], bool (&rok)[NY + 2]) {
#pragma unroll
    for (int k = 0; k < 4; ++k) cok[k] = !kBorder || (unsigned)(bx + k) < (unsigned)w;
#pragma unroll
    for (int k = 0; k < NY + 2; ++k) rok[k] = !kBorder || (unsigned)(by + k) < (unsigned)h;
#pragma unroll
    for (int r = 0; r < NY + 2; ++r) {
        const int yy = kBorder ? clampi(by + r, 0, h - 1) : by + r;
        const uint16_t *row = fr + (size_t)yy * pitch;
#pragma unroll
        for (int c = 0; c < 4; ++c) rv[r][c] = (float)HMFSR_LDG(row + (kBorder ? clampi(bx + c, 0, w - 1) : bx + c));
    }
}

// One frame's contribution to the block's 2 x NY pixels.  rv: the raw block; om: where each
// pixel's Omega comes from; dxs / dys: offsets of the window's columns / rows from
// x0 + v, sqx / sqy their squares; cok / rok: per block column / row, inside the frame
// (kBorder; samples outside are left out); rh: per pixel Rhat; bx, by: the block's first
// sample (its parities give every window's Bayer arrangement).
template <bool kBorder, int NY>
__device__ __forceinline__ void quad_frame(const float (&rv)[NY + 2][4], const QuadOmega<NY> &om, const float (&dxs)[3],
                                           const float (&dys)[3], const float (&sqx)[3], const float (&sqy)[3],
                                           const bool (&cok)[4], const bool (&rok)[NY + 2], const float (&rh)[2 * NY],
                                           int bx, int by, PixelAcc (&acc)[2 * NY]) {
#pragma unroll
    for (int p = 0; p < 2 * NY; ++p) {
        // a rejected frame adds nothing to this pixel
        if (!(rh[p] > 0.f)) continue;
        const int pa = p & 1, pb = p >> 1;
        float Bxx, Byy, Bxy2;
        quad_omega<kBorder, NY>(om, pa, pb, Bxx, Byy, Bxy2);
        float Ax[3], Ex[3], Cy[3];
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            Ax[i] = Bxx * sqx[i];
            Ex[i] = Bxy2 * dxs[i];
            Cy[i] = Byy * sqy[i];
        }
        float w3[3][3];
        bool ok[3][3];
#pragma unroll
        for (int j = 0; j < 3; ++j)
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                w3[j][i] = rv[pb + j][pa + i];
                ok[j][i] = !kBorder || (cok[pa + i] && rok[pb + j]);
            }
        // the window's centre sample (kx, ky) = (bx + pa + 1, by + pb + 1)
        const int cx = (bx + pa + 1) & 1, cy = (by + pb + 1) & 1;
        accumulate_frame_parts<kBorder>(Ax, Ex, Cy, dys, w3, ok, rh[p], (cx ^ cy) != 0, cy != 0, acc[p]);
    }
}

// All frames of the block with top-left output pixel (X, Y) at scale 1 (X even; Y even
// when NY = 2): the arithmetic of merge_px at scale 1, with the sharing described above.
template <bool kDen, int NY, bool kChunk = false>
__device__ __forceinline__ void merge_quad1(const uint16_t *__restrict__ burst, const int4 *__restrict__ geo,
                                            const Geom &g, const float4 *__restrict__ kern,
                                            const float *__restrict__ rhat_planes, float *__restrict__ rgb,
                                            float *__restrict__ den_out, int X, int Y,
                                            const ChunkIO &io = ChunkIO{}) {
    const int ho = g.h, wo = g.w;
    if (X >= wo || Y >= ho) return;  // both sizes are even: a block is wholly inside or outside
    const int u = X >> 1;
    const int txi = min(X / g.tile, g.tx - 1), tyi = min(Y / g.tile, g.ty - 1);
    const size_t hw = (size_t)g.hh * g.wh, ntl = (size_t)g.ty * g.tx;
    const int4 *geo_q = geo + (size_t)tyi * g.tx + txi;
    // Rhat on the base half-res grid at (x0 - 1/2)/2: pixel column pa takes texel columns
    // u - 1 + pa and u + pa at fractions 3/4 (pa = 0) and 1/4 (pa = 1); pixel row Y + pb
    // takes rows ry(Y + pb) and ry + 1 with ry(y) = floor((2 y - 1)/4), fraction
    // ((2 y - 1) mod 4)/4 (clamped reads)
    const int ry0 = (2 * Y - 1) >> 2;
    int rc[3], rr[NY + 1];
#pragma unroll
    for (int k = 0; k < 3; ++k) rc[k] = clampi(u - 1 + k, 0, g.wh - 1);
#pragma unroll
    for (int k = 0; k <= NY; ++k) rr[k] = clampi(ry0 + k, 0, g.hh - 1) * g.wh;
    auto rhat_at = [&](int f, float (&rh)[2 * NY]) {
        if (f == g.ref) {
#pragma unroll
            for (int p = 0; p < 2 * NY; ++p) rh[p] = 1.f;
            return;
        }
        const float *Rp = rhat_planes + (size_t)f * hw;
        float R[NY + 1][3];
#pragma unroll
        for (int j = 0; j <= NY; ++j)
#pragma unroll
            for (int i = 0; i < 3; ++i) R[j][i] = HMFSR_LDG(Rp + rr[j] + rc[i]);
#pragma unroll
        for (int p = 0; p < 2 * NY; ++p) {
            const int pa = p & 1, pb = p >> 1;
            // row ry(Y + pb) is rr[pb] when NY = 2 (Y even); when NY = 1 it is rr[0]
            const float rfx = pa ? 0.25f : 0.75f;
            const float rfy = (float)((2 * (Y + pb) - 1) & 3) * 0.25f;
            const float rw00 = (1.f - rfx) * (1.f - rfy), rw10 = rfx * (1.f - rfy), rw01 = (1.f - rfx) * rfy,
                        rw11 = rfx * rfy;
            rh[p] = fmaf(rw00, R[pb][pa], fmaf(rw10, R[pb][pa + 1], fmaf(rw01, R[pb + 1][pa], rw11 * R[pb + 1][pa + 1])));
        }
    };

    PixelAcc acc[2 * NY];
    const size_t fstride = (size_t)g.h * g.pitch;
    int it0 = 0;
    if constexpr (kChunk) {
        if (io.state_in) {
#pragma unroll
            for (int p = 0; p < 2 * NY; ++p) load_state(io, (size_t)(Y + (p >> 1)) * wo + X + (p & 1), acc[p]);
        }
        it0 = io.skip_base ? 1 : 0;
    }
    // frames in the order base frame, then the others.  Each frame's geometry and Rhat are
    // read at the top of its own iteration: fetching the next frame's a frame ahead held 8
    // more registers through the loop, spilled, and measured 2.5% slower at 12 MP x 8
    int f_nx = kChunk ? frame_of_step(it0, g.ref) : g.ref;
    for (int it = it0; it < g.n; ++it) {
        const int f = f_nx;
        const int4 gq = HMFSR_LDG(geo_q + (size_t)f * ntl);
        float rh[2 * NY];
        rhat_at(f, rh);
        if (it + 1 < g.n) f_nx = (it + 1 <= g.ref) ? it : it + 1;
        bool any = false;
#pragma unroll
        for (int p = 0; p < 2 * NY; ++p) any |= rh[p] > 0.f;
        if (!any) continue;  // every pixel rejected this frame
        // geometry (Q = 2): F = floor(2 v), z = 2 v - F; window centre kx = X + Kx with
        // Kx = floor((F + 1) / 2) = round(v) (ties up); centre offset (2 Kx - F - z) / 2
        const int FX = gq.x, FY = gq.y;
        const float zx = __int_as_float(gq.z), zy = __int_as_float(gq.w);
        const int Kx = (FX + 1) >> 1, Ky = (FY + 1) >> 1;
        const float dx0 = ((float)(2 * Kx - FX) - zx) * 0.5f;
        const float dy0 = ((float)(2 * Ky - FY) - zy) * 0.5f;
        const float dxs[3] = {dx0 - 1.f, dx0, dx0 + 1.f};
        const float dys[3] = {dy0 - 1.f, dy0, dy0 + 1.f};
        float sqx[3], sqy[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            sqx[k] = dxs[k] * dxs[k];
            sqy[k] = dys[k] * dys[k];
        }
        // Omega sampling (frame f's half-res grid at (x0 + v - 1/2)/2): output column x
        // samples at (2 x - 1 + F + z)/4, i.e. cell (2 x - 1 + F) div 4, fraction
        // (((2 x - 1 + F) mod 4) + z)/4
        QuadOmega<NY> om;
        om.K = kern + (size_t)f * hw;
        om.wh = g.wh;
        om.hh = g.hh;
        om.u = u;
        om.v = 0;
#pragma unroll
        for (int pa = 0; pa < 2; ++pa) {
            const int gx = 2 * pa - 1 + FX;  // relative to 2 X = 4 u
            om.Ox[pa] = gx >> 2;
            om.fx[pa] = ((float)(gx & 3) + zx) * 0.25f;
        }
#pragma unroll
        for (int pb = 0; pb < NY; ++pb) {
            const int gy = 2 * (Y + pb) - 1 + FY;  // absolute
            om.Oy[pb] = gy >> 2;
            om.fy[pb] = ((float)(gy & 3) + zy) * 0.25f;
        }
        const int bx = X + Kx - 1, by = Y + Ky - 1;  // first sample of the raw block
        const uint16_t *fr = burst + (size_t)f * fstride;
        const bool inside = (unsigned)bx <= (unsigned)(g.w - 4) && (unsigned)by <= (unsigned)(g.h - NY - 2) &&
                            u + om.Ox[0] >= 0 && u + om.Ox[1] + 1 < g.wh && om.Oy[0] >= 0 &&
                            om.Oy[NY - 1] + 1 < g.hh;
        float rv[NY + 2][4];
        bool cok[4], rok[NY + 2];
        if (inside) {
            quad_block<false, NY>(fr, g.pitch, g.h, g.w, bx, by, rv, cok, rok);
            quad_frame<false, NY>(rv, om, dxs, dys, sqx, sqy, cok, rok, rh, bx, by, acc);
        } else {
            quad_block<true, NY>(fr, g.pitch, g.h, g.w, bx, by, rv, cok, rok);
            quad_frame<true, NY>(rv, om, dxs, dys, sqx, sqy, cok, rok, rh, bx, by, acc);
        }
    }
    const size_t po = (size_t)ho * wo;
    if constexpr (kChunk) {
        if (io.state_out) {
#pragma unroll
            for (int p = 0; p < 2 * NY; ++p) store_state(io, (size_t)(Y + (p >> 1)) * wo + X + (p & 1), acc[p]);
            return;
        }
    }
#pragma unroll
    for (int pb = 0; pb < NY; ++pb) {
        const size_t o = (size_t)(Y + pb) * wo + X;
        const PixelAcc &a0 = acc[2 * pb], &a1 = acc[2 * pb + 1];
        HMFSR_ST(reinterpret_cast<float2 *>(rgb + o), make_float2(a0.numR / a0.denR, a1.numR / a1.denR));
        HMFSR_ST(reinterpret_cast<float2 *>(rgb + po + o), make_float2(a0.numG / a0.denG, a1.numG / a1.denG));
        HMFSR_ST(reinterpret_cast<float2 *>(rgb + 2 * po + o), make_float2(a0.numB / a0.denB, a1.numB / a1.denB));
        if (kDen) {
            HMFSR_ST(reinterpret_cast<float2 *>(den_out + o), make_float2(log2f(a0.denR) - a0.mR, log2f(a1.denR) - a1.mR));
            HMFSR_ST(reinterpret_cast<float2 *>(den_out + po + o),
                     make_float2(log2f(a0.denG) - a0.mG, log2f(a1.denG) - a1.mG));
            HMFSR_ST(reinterpret_cast<float2 *>(den_out + 2 * po + o),
                     make_float2(log2f(a0.denB) - a0.mB, log2f(a1.denB) - a1.mB));
        }
    }
}

}  // namespace stage
}  // namespace hmfsr
