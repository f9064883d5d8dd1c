/*
 * FP64 oracle for the handheld multi-frame super-resolution merge and tile alignment
 * (Wronski et al. 2019).  TEST INFRASTRUCTURE ONLY: a plain, slow CPU restatement of the
 * paper's equations, used to check the CUDA path; it shares no code with that path.
 *
 * Every function evaluates the paper's definitions literally, per pixel, in double
 * precision.  Where the paper is silent or ambiguous, the reading taken is stated at the
 * place it is used.  Build: gcc -O2 -ffp-contract=off -fopenmp (no fast-math), so that
 * the FP64 decisions (motion-prior threshold, alignment conditioning guard) are the plain
 * IEEE operation sequence written here.
 *
 * Parity notes (pins live in tests/): every function below is pinned by at least one
 * property test; none is "parity unpinned".
 */
#include "hmfsr_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------------------ */
/* small helpers                                                                         */
/* ------------------------------------------------------------------------------------ */
static inline int clampi(int x, int lo, int hi) { return x < lo ? lo : (x > hi ? hi : x); }
static inline double clampd(double x, double lo, double hi) { return x < lo ? lo : (x > hi ? hi : x); }
static inline long long floor_div(long long a, long long b) /* b > 0 */
{
    long long q = a / b;
    if ((a % b) != 0 && a < 0) q -= 1;
    return q;
}

static void set_threads(int n_threads)
{
#ifdef _OPENMP
    if (n_threads > 0) omp_set_num_threads(n_threads);
#else
    (void)n_threads;
#endif
}

/* CFA channel of raw pixel (x, y): RGGB -> 0 R, 1 G, 2 B. */
static inline int cfa_channel(int x, int y) { return (x & 1) + (y & 1); }

/* ------------------------------------------------------------------------------------ */
/* Half-res luminance and guide image (Sec. 5.1.2; Sec. 5.2.2)                          */
/* ------------------------------------------------------------------------------------ */
/* Lq = R + G1 + G2 + B of the quad.  The paper says the four channels of a Bayer quad
 * are combined into one luminance pixel without saying how; the plain sum is used. */
static inline int32_t luma_at(const uint16_t *raw, int h, int w, int u, int v)
{
    int hh = h / 2, wh = w / 2;
    u = clampi(u, 0, wh - 1);
    v = clampi(v, 0, hh - 1);
    const uint16_t *r0 = raw + (size_t)(2 * v) * w + 2 * u;
    const uint16_t *r1 = r0 + w;
    return (int32_t)r0[0] + r0[1] + r1[0] + r1[1];
}

/* Guide pixel (Sec. 5.2.2): R and B as they are, green = average of the two greens.
 * Returned as integers: c = 0 -> R, 1 -> G1 + G2 (twice the guide's green), 2 -> B. */
static inline int32_t guide_at(const uint16_t *raw, int h, int w, int u, int v, int c)
{
    int hh = h / 2, wh = w / 2;
    u = clampi(u, 0, wh - 1);
    v = clampi(v, 0, hh - 1);
    const uint16_t *r0 = raw + (size_t)(2 * v) * w + 2 * u;
    const uint16_t *r1 = r0 + w;
    if (c == 0) return r0[0];
    if (c == 1) return (int32_t)r0[1] + r1[0];
    return r1[1];
}

int orc_luma(const uint16_t *raw, int h, int w, int32_t *lq)
{
    if (!raw || !lq || h < 2 || w < 2 || (h & 1) || (w & 1)) return -1;
    int hh = h / 2, wh = w / 2;
    for (int v = 0; v < hh; ++v)
        for (int u = 0; u < wh; ++u) lq[(size_t)v * wh + u] = luma_at(raw, h, w, u, v);
    return 0;
}

/* ------------------------------------------------------------------------------------ */
/* Structure tensor (Eq. 3)                                                              */
/* ------------------------------------------------------------------------------------ */
/* Reading of "finite forward differencing in a 3x3 window giving four horizontal and
 * vertical gradient values": the 3x3 half-res window centred on (u,v) holds four 2x2
 * sub-squares with top-left corners (u+i, v+j), i, j in {-1, 0}.  Each sub-square gives
 * one forward-difference gradient (the sum of its two horizontal, resp. vertical,
 * differences); the tensor sums the four outer products.  Reads clamp at the border.
 * Exact in int64. */
static void tensor_at(const uint16_t *raw, int h, int w, int u, int v, int64_t *a, int64_t *b, int64_t *c)
{
    int64_t sa = 0, sb = 0, sc = 0;
    for (int j = -1; j <= 0; ++j)
        for (int i = -1; i <= 0; ++i) {
            int64_t l00 = luma_at(raw, h, w, u + i, v + j);
            int64_t l10 = luma_at(raw, h, w, u + i + 1, v + j);
            int64_t l01 = luma_at(raw, h, w, u + i, v + j + 1);
            int64_t l11 = luma_at(raw, h, w, u + i + 1, v + j + 1);
            int64_t gx = (l10 - l00) + (l11 - l01);
            int64_t gy = (l01 - l00) + (l11 - l10);
            sa += gx * gx;
            sb += gx * gy;
            sc += gy * gy;
        }
    *a = sa; *b = sb; *c = sc;
}

int orc_structure_tensor(const uint16_t *raw, int h, int w, int u, int v, int64_t out[3])
{
    if (!raw || !out || h < 2 || w < 2) return -1;
    tensor_at(raw, h, w, u, v, &out[0], &out[1], &out[2]);
    return 0;
}

/* ------------------------------------------------------------------------------------ */
/* Kernel covariance (Eq. 4 with the supplement's kernel-shape heuristics)               */
/* ------------------------------------------------------------------------------------ */
/* Eigen-analysis of [[a, b], [b, c]]: lambda_{1,2} = (tr +- r)/2 with
 * r = sqrt((a-c)^2 + 4 b^2); the dominant eigenvector e1 is at angle theta with
 * cos 2theta = (a-c)/r, sin 2theta = 2b/r.  When a == c and b == 0 the direction is
 * undefined; the reading taken is theta = 0 (e1 = x axis).
 *
 * Heuristics (supplement S.1): A = 1 + sqrt((l1-l2)/(l1+l2)) (A = 1 when l1+l2 = 0);
 * D = clamp(1 - sqrt(l1)/D_tr + D_th, 0, 1), printed formula taken literally, with l1 in
 * units of the luminance normalised to [0,1]: one forward-difference gradient of the sum
 * luminance spans 2 pixel differences of 4 samples, so g_norm = g / (8 WL), and the
 * tensor is the mean over its four gradients, l_norm = l / (4 (8 WL)^2).
 * k^_stretch = k_detail * k_stretch * A, k^_shrink = k_detail / (k_shrink * A), and
 * k_i = ((1-D) k^_i + D k_detail k_denoise)^2 (variances, raw px^2).
 *
 * Reading of Eq. 4's assignment: the text stretches kernels ALONG edges, i.e. along
 * e2 (perpendicular to the dominant gradient), so the stretched variance goes on e2 and
 * the shrunk one on e1:  Omega = k_across e1 e1^T + k_along e2 e2^T. */
static void kernel_from_tensor(int64_t a, int64_t b, int64_t c, const orc_params *p, int wl, double out[11])
{
    int64_t tr_i = a + c;
    double amc = (double)(a - c);
    double r = sqrt(amc * amc + 4.0 * (double)b * (double)b);
    double tr = (double)tr_i;
    double l1 = 0.5 * (tr + r), l2 = 0.5 * (tr - r);
    double cs, sn;
    if (a == c && b == 0) { cs = 1.0; sn = 0.0; }
    else { cs = amc / r; sn = 2.0 * (double)b / r; }
    double A = (tr_i == 0) ? 1.0 : 1.0 + sqrt(r / tr);
    double norm = 4.0 * (8.0 * wl) * (8.0 * wl);
    double l1n = l1 / norm;
    double D = clampd(1.0 - sqrt(l1n) / p->d_tr + p->d_th, 0.0, 1.0);
    double kh_along = p->k_detail * (p->k_stretch * A);
    double kh_across = p->k_detail / (p->k_shrink * A);
    double kd = p->k_detail * p->k_denoise;
    double k_along = (1.0 - D) * kh_along + D * kd;
    double k_across = (1.0 - D) * kh_across + D * kd;
    k_along *= k_along;
    k_across *= k_across;
    /* e1 e1^T = 1/2 [[1+cs, sn], [sn, 1-cs]],  e2 e2^T = I - e1 e1^T */
    double e1xx = 0.5 * (1.0 + cs), e1xy = 0.5 * sn, e1yy = 0.5 * (1.0 - cs);
    out[0] = k_across * e1xx + k_along * (1.0 - e1xx);
    out[1] = k_across * e1xy - k_along * e1xy;
    out[2] = k_across * e1yy + k_along * (1.0 - e1yy);
    out[3] = l1; out[4] = l2; out[5] = A; out[6] = D;
    out[7] = k_along; out[8] = k_across; out[9] = cs; out[10] = sn;
}

int orc_kernel_from_tensor(int64_t a, int64_t b, int64_t c, const orc_params *p, int wl, double out[11])
{
    if (!p || !out || wl <= 0) return -1;
    kernel_from_tensor(a, b, c, p, wl, out);
    return 0;
}

static void omega_at(const uint16_t *raw, int h, int w, int u, int v, const orc_params *p, int wl, double om[3])
{
    int64_t a, b, c;
    double k[11];
    tensor_at(raw, h, w, u, v, &a, &b, &c);
    kernel_from_tensor(a, b, c, p, wl, k);
    om[0] = k[0]; om[1] = k[1]; om[2] = k[2];
}

int orc_omega_plane(const uint16_t *raw, int h, int w, const orc_params *p, int wl, double *omega)
{
    if (!raw || !p || !omega || h < 2 || w < 2 || (h & 1) || (w & 1)) return -1;
    int hh = h / 2, wh = w / 2;
    size_t plane = (size_t)hh * wh;
#pragma omp parallel for schedule(static)
    for (int v = 0; v < hh; ++v)
        for (int u = 0; u < wh; ++u) {
            double om[3];
            omega_at(raw, h, w, u, v, p, wl, om);
            for (int k = 0; k < 3; ++k) omega[k * plane + (size_t)v * wh + u] = om[k];
        }
    return 0;
}

/* ------------------------------------------------------------------------------------ */
/* Motion prior (Eq. 7-8)                                                                */
/* ------------------------------------------------------------------------------------ */
/* M = sqrt(Mx^2 + My^2), Mx / My = max - min of the tile vectors over the 3x3 tile
 * neighbourhood (tiles outside the grid are left out); s = s1 if M > M_th else s2. */
static double tile_M(const float *motion, int ty, int tx, int y, int x)
{
    double mnx = INFINITY, mxx = -INFINITY, mny = INFINITY, mxy = -INFINITY;
    for (int j = -1; j <= 1; ++j)
        for (int i = -1; i <= 1; ++i) {
            int yy = y + j, xx = x + i;
            if (yy < 0 || yy >= ty || xx < 0 || xx >= tx) continue;
            const float *mv = motion + ((size_t)yy * tx + xx) * 2;
            double vx = (double)mv[0], vy = (double)mv[1];
            if (vx < mnx) mnx = vx;
            if (vx > mxx) mxx = vx;
            if (vy < mny) mny = vy;
            if (vy > mxy) mxy = vy;
        }
    double Mx = mxx - mnx, My = mxy - mny;
    double sq = Mx * Mx + My * My;
    return sqrt(sq);
}

int orc_tile_strength(const float *motion, int ty, int tx, const orc_params *p, double *M, double *s)
{
    if (!motion || !p || ty <= 0 || tx <= 0) return -1;
    for (int y = 0; y < ty; ++y)
        for (int x = 0; x < tx; ++x) {
            double m = tile_M(motion, ty, tx, y, x);
            if (M) M[(size_t)y * tx + x] = m;
            if (s) s[(size_t)y * tx + x] = (m > p->m_th) ? p->s1 : p->s2;
        }
    return 0;
}

/* ------------------------------------------------------------------------------------ */
/* Robustness (Eq. 5, 6, 9; Sec. 5.2.2)                                                  */
/* ------------------------------------------------------------------------------------ */
/* 3x3 box sum of a guide channel (clamped reads); `sq` selects the sum of squares. */
static int64_t box_sum(const uint16_t *raw, int h, int w, int u, int v, int c, int sq)
{
    int64_t s = 0;
    for (int j = -1; j <= 1; ++j)
        for (int i = -1; i <= 1; ++i) {
            int64_t g = guide_at(raw, h, w, u + i, v + j, c);
            s += sq ? g * g : g;
        }
    return s;
}

/* Guide-channel 3x3 mean of frame `raw` at (u,v), in DN of the guide image (green =
 * average of the two greens).  The local-mean image is defined on the half-res grid;
 * a read outside it takes the nearest pixel of that image (clamped read). */
static double box_mean(const uint16_t *raw, int h, int w, int u, int v, int c)
{
    u = clampi(u, 0, w / 2 - 1);
    v = clampi(v, 0, h / 2 - 1);
    double s = (double)box_sum(raw, h, w, u, v, c, 0);
    return (c == 1) ? s / 18.0 : s / 9.0;
}

/* Bilinear sample of the 3x3 mean of frame `raw` at continuous half-res (fx, fy);
 * reads clamp at the border. */
static double mean_bilinear(const uint16_t *raw, int h, int w, double fx, double fy, int c)
{
    double x0 = floor(fx), y0 = floor(fy);
    double ax = fx - x0, ay = fy - y0;
    int ix = (int)x0, iy = (int)y0;
    double m00 = box_mean(raw, h, w, ix, iy, c);
    double m10 = box_mean(raw, h, w, ix + 1, iy, c);
    double m01 = box_mean(raw, h, w, ix, iy + 1, c);
    double m11 = box_mean(raw, h, w, ix + 1, iy + 1, c);
    return (1.0 - ay) * ((1.0 - ax) * m00 + ax * m10) + ay * ((1.0 - ax) * m01 + ax * m11);
}

typedef struct {
    int h, w, tile, ty, tx, wl;
    const orc_params *p;
} rob_geom;

/* Statistical robustness R at base half-res pixel (u,v) for frame `alt`.
 * Readings taken where the paper is silent:
 *  - sigma_ms (local spatial std) comes from the base frame; the local means of both
 *    frames are compared, the aligned frame's mean being sampled bilinearly at the
 *    position displaced by the tile's vector (v/2 in half-res px).  The tile is the one
 *    holding the half-res pixel: floor(2u / tile).
 *  - noise model: the paper tabulates sigma_md and d_md by Monte Carlo; here the closed
 *    form for the linear model var(x) = a x + b at x = clamp(mu_base, 0, WL) is used,
 *    halved for the green guide channel (mean of two samples): sigma_md = sqrt(var),
 *    d_md = sqrt(2 var / 9) (difference of two 9-sample means).
 *  - the colour difference and sigma are vectors over (R, G, B); the ratio in Eq. 5 is
 *    |d|^2 / max(|sigma|^2, 1e-12 WL^2).
 *  - R is clamped to [0, 1] (a weight of one merges fully, zero rejects). */
/* Modelled statistics of one guide channel at brightness mu (Eq. 6): the variance
 * sigma_md^2 expected of a 3x3 patch of constant brightness and d_md^2, the expected
 * squared difference of two such patches' means.  Closed form (var = a x + b per raw
 * sample, halved for the green mean of two; d_md^2 = 2 var / 9), or the Monte-Carlo table
 * interpolated linearly between brightness levels. */
static void modelled_stats(const orc_params *p, int wl, double mu, int c, double *var_md, double *dmd2)
{
    if (p->noise_table) {
        double t = clampd(mu, 0.0, (double)wl) * (double)(ORC_NOISE_LEVELS - 1) / (double)wl;
        int i = (int)floor(t);
        if (i > ORC_NOISE_LEVELS - 2) i = ORC_NOISE_LEVELS - 2;
        double f = t - (double)i;
        int k = (c == 1) ? 1 : 0;
        const double *a = p->noise_table + 4 * i, *b = a + 4;
        *var_md = (1.0 - f) * a[k] + f * b[k];
        *dmd2 = (1.0 - f) * a[2 + k] + f * b[2 + k];
        return;
    }
    double gs = (c == 1) ? 2.0 : 1.0;
    double v = (p->noise_a * clampd(mu, 0.0, (double)wl) + p->noise_b) / gs;
    if (v < 0.0) v = 0.0;
    *var_md = v;
    *dmd2 = 2.0 * v / 9.0;
}

/* High-frequency artifact test (supplement, High Frequency Artifacts Removal) at base
 * texel (u, v): the local variance lost to the low-pass.  "Before" is the 3x3 population
 * variance of the guide, summed over R, G, B; "after" is the population variance of the
 * 3x3 local means over the 3x3 texels around (u, v) (clamped to the grid).  With the
 * green guide at half scale, 4 x both variances times 81 and 6561 are the exact integers
 * B = sum_c w_c (9 S2 - S1^2) and A = sum_c w_c (9 sum_k S1_k^2 - (sum_k S1_k)^2),
 * w = (4, 1, 4): the loss is A < kappa 81 B, decided in FP64 from exact integers. */
static int hf_loss_at(const uint16_t *base, int h, int w, int u, int v, double kappa)
{
    static const int64_t wgt[3] = {4, 1, 4};
    int64_t A = 0, B = 0;
    for (int c = 0; c < 3; ++c) {
        int64_t s1 = box_sum(base, h, w, u, v, c, 0), s2 = box_sum(base, h, w, u, v, c, 1);
        B += wgt[c] * (9 * s2 - s1 * s1);
        int64_t t1 = 0, t2 = 0;
        for (int j = -1; j <= 1; ++j)
            for (int i = -1; i <= 1; ++i) {
                int64_t m = box_sum(base, h, w, clampi(u + i, 0, w / 2 - 1), clampi(v + j, 0, h / 2 - 1), c, 0);
                t1 += m;
                t2 += m * m;
            }
        A += wgt[c] * (9 * t2 - t1 * t1);
    }
    return B > 0 && (double)A < kappa * (81.0 * (double)B);
}

static double robustness_at(const uint16_t *base, const uint16_t *alt, const float *motion_alt,
                            const double *s_tile, const rob_geom *g, int u, int v)
{
    const orc_params *p = g->p;
    int tyi = clampi((2 * v) / g->tile, 0, g->ty - 1);
    int txi = clampi((2 * u) / g->tile, 0, g->tx - 1);
    /* high-frequency regions with a large local motion span are rejected outright */
    if (p->hf_loss > 0.0 && tile_M(motion_alt, g->ty, g->tx, tyi, txi) > p->m_th &&
        hf_loss_at(base, g->h, g->w, u, v, p->hf_loss))
        return 0.0;
    const float *mv = motion_alt + ((size_t)tyi * g->tx + txi) * 2;
    double fx = (double)u + 0.5 * (double)mv[0];
    double fy = (double)v + 0.5 * (double)mv[1];
    double dd = 0.0, ss = 0.0;
    for (int c = 0; c < 3; ++c) {
        double s1 = (double)box_sum(base, g->h, g->w, u, v, c, 0);
        double s2 = (double)box_sum(base, g->h, g->w, u, v, c, 1);
        double gs = (c == 1) ? 2.0 : 1.0; /* green guide = (G1 + G2) / 2 */
        double mu = s1 / (9.0 * gs);
        double var_ms = (9.0 * s2 - s1 * s1) / (81.0 * gs * gs);
        if (var_ms < 0.0) var_ms = 0.0;
        double sigma_ms = sqrt(var_ms);
        double mu_n = mean_bilinear(alt, g->h, g->w, fx, fy, c);
        double d_ms = mu - mu_n;
        double var_md, dmd2;
        modelled_stats(p, g->wl, mu, c, &var_md, &dmd2);
        double sigma_md = sqrt(var_md);
        double sigma = sigma_ms > sigma_md ? sigma_ms : sigma_md;       /* Eq. 6 */
        double den = d_ms * d_ms + dmd2;
        double d = den > 0.0 ? d_ms * (d_ms * d_ms) / den : 0.0;        /* Eq. 6 */
        dd += d * d;
        ss += sigma * sigma;
    }
    double eps = 1e-12 * (double)g->wl * (double)g->wl;
    double ratio = dd / (ss > eps ? ss : eps);
    double s = s_tile[(size_t)tyi * g->tx + txi];
    return clampd(s * exp(-ratio) - p->t, 0.0, 1.0);                     /* Eq. 5 */
}

/* Rhat = min of R over the 5x5 window of valid pixels (Eq. 9). */
static double rhat_from_R(const double *R, int hh, int wh, int u, int v)
{
    double m = INFINITY;
    for (int j = -2; j <= 2; ++j)
        for (int i = -2; i <= 2; ++i) {
            int uu = u + i, vv = v + j;
            if (uu < 0 || uu >= wh || vv < 0 || vv >= hh) continue;
            double r = R[(size_t)vv * wh + uu];
            if (r < m) m = r;
        }
    return m;
}

int orc_robustness(const uint16_t *base, const uint16_t *alt, int h, int w, const float *motion_alt,
                   int tile, const orc_params *p, int wl, double *R, double *Rhat)
{
    if (!base || !alt || !motion_alt || !p || h < 2 || w < 2 || (h & 1) || (w & 1) || tile < 2 || (tile & 1))
        return -1;
    int hh = h / 2, wh = w / 2;
    rob_geom g = { h, w, tile, (h + tile - 1) / tile, (w + tile - 1) / tile, wl, p };
    double *s_tile = (double *)malloc(sizeof(double) * (size_t)g.ty * g.tx);
    double *Rb = R ? R : (double *)malloc(sizeof(double) * (size_t)hh * wh);
    if (!s_tile || !Rb) { free(s_tile); if (!R) free(Rb); return -2; }
    orc_tile_strength(motion_alt, g.ty, g.tx, p, NULL, s_tile);
#pragma omp parallel for schedule(static)
    for (int v = 0; v < hh; ++v)
        for (int u = 0; u < wh; ++u) Rb[(size_t)v * wh + u] = robustness_at(base, alt, motion_alt, s_tile, &g, u, v);
    if (Rhat) {
#pragma omp parallel for schedule(static)
        for (int v = 0; v < hh; ++v)
            for (int u = 0; u < wh; ++u) Rhat[(size_t)v * wh + u] = rhat_from_R(Rb, hh, wh, u, v);
    }
    free(s_tile);
    if (!R) free(Rb);
    return 0;
}

/* ------------------------------------------------------------------------------------ */
/* Merge (Eq. 1-2)                                                                       */
/* ------------------------------------------------------------------------------------ */
/* Per-frame data for the merge: Omega and Rhat on half-res rows [r0, r1) (NULL planes
 * mean "evaluate on demand"). */
typedef struct {
    const uint16_t *burst;
    int n, h, w, ref, tile, ty, tx, wl;
    const float *motion;
    const orc_params *p;
    /* per frame, rows [om_r0[f], om_r1[f]) of Omega [3][rows][wh] */
    double **om;
    int *om_r0, *om_r1;
    /* per frame, rows [rh_r0[f], rh_r1[f]) of Rhat [rows][wh] (base grid) */
    double **rh;
    int *rh_r0, *rh_r1;
    double **s_tile;
} merge_ctx;

static inline const uint16_t *frame_ptr(const merge_ctx *m, int f) { return m->burst + (size_t)f * m->h * m->w; }
static inline const float *motion_ptr(const merge_ctx *m, int f) { return m->motion + (size_t)f * m->ty * m->tx * 2; }

static void omega_get(const merge_ctx *m, int f, int u, int v, double om[3])
{
    int hh = m->h / 2, wh = m->w / 2;
    u = clampi(u, 0, wh - 1);
    v = clampi(v, 0, hh - 1);
    if (m->om && m->om[f] && v >= m->om_r0[f] && v < m->om_r1[f]) {
        size_t rows = (size_t)(m->om_r1[f] - m->om_r0[f]);
        const double *pl = m->om[f] + (size_t)(v - m->om_r0[f]) * wh + u;
        om[0] = pl[0]; om[1] = pl[rows * wh]; om[2] = pl[2 * rows * wh];
        return;
    }
    omega_at(frame_ptr(m, f), m->h, m->w, u, v, m->p, m->wl, om);
}

static double rhat_get(const merge_ctx *m, int f, int u, int v)
{
    int hh = m->h / 2, wh = m->w / 2;
    u = clampi(u, 0, wh - 1);
    v = clampi(v, 0, hh - 1);
    if (m->rh && m->rh[f] && v >= m->rh_r0[f] && v < m->rh_r1[f])
        return m->rh[f][(size_t)(v - m->rh_r0[f]) * wh + u];
    /* on demand: min over the 5x5 window of R */
    rob_geom g = { m->h, m->w, m->tile, m->ty, m->tx, m->wl, m->p };
    double best = INFINITY;
    for (int j = -2; j <= 2; ++j)
        for (int i = -2; i <= 2; ++i) {
            int uu = u + i, vv = v + j;
            if (uu < 0 || uu >= wh || vv < 0 || vv >= hh) continue;
            double r = robustness_at(frame_ptr(m, m->ref), frame_ptr(m, f), motion_ptr(m, f), m->s_tile[f], &g, uu, vv);
            if (r < best) best = r;
        }
    return best;
}

/* Output-pixel geometry.  Reading of the (unstated) resampling grid: pixel centres at
 * integers on both grids, so output pixel X sits at raw x0 = (X + 1/2)/s - 1/2, written
 * exactly as the rational P/Q with P = 2 den X + den - num and Q = 2 num. */
static void merge_pixel(const merge_ctx *m, int snum, int sden, int X, int Y, double out[3], double den_out[3])
{
    const long long Q = 2LL * snum;
    const long long Px = 2LL * sden * X + sden - snum;
    const long long Py = 2LL * sden * Y + sden - snum;
    const double x0 = (double)Px / (double)Q, y0 = (double)Py / (double)Q;
    /* tile of the output pixel on the base frame (motion is constant per tile) */
    int txi = (int)floor_div(Px, Q * m->tile);
    int tyi = (int)floor_div(Py, Q * m->tile);
    txi = clampi(txi, 0, m->tx - 1);
    tyi = clampi(tyi, 0, m->ty - 1);
    double num[3] = { 0, 0, 0 }, den[3] = { 0, 0, 0 };
    for (int f = 0; f < m->n; ++f) {
        double vx = 0.0, vy = 0.0;
        if (f != m->ref) {
            const float *mv = motion_ptr(m, f) + ((size_t)tyi * m->tx + txi) * 2;
            vx = (double)mv[0];
            vy = (double)mv[1];
        }
        /* 3x3 window centre: the raw pixel nearest to x0 + v (ties round up), computed
         * exactly: floor((P + Q/2 + Q v) / Q) with Q v exact in FP64. */
        long long kx = floor_div(Px + Q / 2 + (long long)floor((double)Q * vx), Q);
        long long ky = floor_div(Py + Q / 2 + (long long)floor((double)Q * vy), Q);
        double px = x0 + vx, py = y0 + vy;
        /* Omega: bilinear on frame f's half-res grid (centre of (u,v) at raw 2u + 1/2) */
        double hx = (px - 0.5) / 2.0, hy = (py - 0.5) / 2.0;
        double fx0 = floor(hx), fy0 = floor(hy);
        double ax = hx - fx0, ay = hy - fy0;
        int ix = (int)fx0, iy = (int)fy0;
        double o00[3], o10[3], o01[3], o11[3], om[3];
        omega_get(m, f, ix, iy, o00);
        omega_get(m, f, ix + 1, iy, o10);
        omega_get(m, f, ix, iy + 1, o01);
        omega_get(m, f, ix + 1, iy + 1, o11);
        for (int k = 0; k < 3; ++k)
            om[k] = (1.0 - ay) * ((1.0 - ax) * o00[k] + ax * o10[k]) + ay * ((1.0 - ax) * o01[k] + ax * o11[k]);
        double det = om[0] * om[2] - om[1] * om[1];
        double ixx = om[2] / det, ixy = -om[1] / det, iyy = om[0] / det;   /* Omega^-1 */
        /* Rhat: bilinear on the base half-res grid at the base position; 1 for the base */
        double rhat = 1.0;
        if (f != m->ref) {
            double gx = (x0 - 0.5) / 2.0, gy = (y0 - 0.5) / 2.0;
            double gx0 = floor(gx), gy0 = floor(gy);
            double bx = gx - gx0, by = gy - gy0;
            int jx = (int)gx0, jy = (int)gy0;
            double r00 = rhat_get(m, f, jx, jy), r10 = rhat_get(m, f, jx + 1, jy);
            double r01 = rhat_get(m, f, jx, jy + 1), r11 = rhat_get(m, f, jx + 1, jy + 1);
            rhat = (1.0 - by) * ((1.0 - bx) * r00 + bx * r10) + by * ((1.0 - bx) * r01 + bx * r11);
        }
        const uint16_t *fr = frame_ptr(m, f);
        /* the nine samples of the 3x3 Bayer neighbourhood; samples outside the frame
         * are left out (the paper does not say) */
        for (int j = -1; j <= 1; ++j)
            for (int i = -1; i <= 1; ++i) {
                long long qx = kx + i, qy = ky + j;
                if (qx < 0 || qx >= m->w || qy < 0 || qy >= m->h) continue;
                double dx = (double)qx - px, dy = (double)qy - py;
                double qf = ixx * dx * dx + 2.0 * ixy * dx * dy + iyy * dy * dy;
                double wgt = exp(-0.5 * qf);                                   /* Eq. 2 */
                int c = cfa_channel((int)qx, (int)qy);
                double cval = (double)fr[(size_t)qy * m->w + qx];
                num[c] += cval * wgt * rhat;                                   /* Eq. 1 */
                den[c] += wgt * rhat;
            }
    }
    for (int c = 0; c < 3; ++c) {
        out[c] = num[c] / den[c];
        if (den_out) den_out[c] = den[c];
    }
}

static void free_ctx(merge_ctx *m)
{
    if (m->om) for (int f = 0; f < m->n; ++f) free(m->om[f]);
    if (m->rh) for (int f = 0; f < m->n; ++f) free(m->rh[f]);
    if (m->s_tile) for (int f = 0; f < m->n; ++f) free(m->s_tile[f]);
    free(m->om); free(m->rh); free(m->s_tile);
    free(m->om_r0); free(m->om_r1); free(m->rh_r0); free(m->rh_r1);
}

static int init_ctx(merge_ctx *m, const uint16_t *burst, int n, int h, int w, int ref, const float *motion,
                    int tile, const orc_params *p, int wl)
{
    memset(m, 0, sizeof(*m));
    if (!burst || !motion || !p || n < 1 || h < 2 || w < 2 || (h & 1) || (w & 1) || ref < 0 || ref >= n ||
        tile < 2 || (tile & 1) || wl <= 0)
        return -1;
    m->burst = burst; m->n = n; m->h = h; m->w = w; m->ref = ref; m->tile = tile;
    m->ty = (h + tile - 1) / tile; m->tx = (w + tile - 1) / tile; m->wl = wl;
    m->motion = motion; m->p = p;
    m->s_tile = (double **)calloc((size_t)n, sizeof(double *));
    if (!m->s_tile) return -2;
    for (int f = 0; f < n; ++f) {
        m->s_tile[f] = (double *)malloc(sizeof(double) * (size_t)m->ty * m->tx);
        if (!m->s_tile[f]) return -2;
        orc_tile_strength(motion_ptr(m, f), m->ty, m->tx, p, NULL, m->s_tile[f]);
    }
    return 0;
}

/* Precompute Omega and Rhat on the half-res rows that output rows [y0, y1) can touch. */
static int precompute_rows(merge_ctx *m, int snum, int sden, int y0, int y1)
{
    int n = m->n, hh = m->h / 2, wh = m->w / 2;
    m->om = (double **)calloc((size_t)n, sizeof(double *));
    m->rh = (double **)calloc((size_t)n, sizeof(double *));
    m->om_r0 = (int *)calloc((size_t)n, sizeof(int)); m->om_r1 = (int *)calloc((size_t)n, sizeof(int));
    m->rh_r0 = (int *)calloc((size_t)n, sizeof(int)); m->rh_r1 = (int *)calloc((size_t)n, sizeof(int));
    if (!m->om || !m->rh || !m->om_r0 || !m->om_r1 || !m->rh_r0 || !m->rh_r1) return -2;
    /* raw rows of the band's base positions */
    double ylo = ((double)y0 + 0.5) * sden / snum - 0.5;
    double yhi = ((double)y1 - 0.5) * sden / snum - 0.5;
    for (int f = 0; f < n; ++f) {
        double vmin = 0.0, vmax = 0.0;
        if (f != m->ref) {
            const float *mv = motion_ptr(m, f);
            vmin = INFINITY; vmax = -INFINITY;
            for (int t = 0; t < m->ty * m->tx; ++t) {
                double vy = mv[2 * t + 1];
                if (vy < vmin) vmin = vy;
                if (vy > vmax) vmax = vy;
            }
        }
        int r0 = (int)floor((ylo + vmin - 0.5) / 2.0) - 2;
        int r1 = (int)ceil((yhi + vmax - 0.5) / 2.0) + 3;
        r0 = clampi(r0, 0, hh); r1 = clampi(r1, 0, hh);
        m->om_r0[f] = r0; m->om_r1[f] = r1;
        if (r1 > r0) {
            size_t rows = (size_t)(r1 - r0);
            m->om[f] = (double *)malloc(sizeof(double) * 3 * rows * wh);
            if (!m->om[f]) return -2;
            const uint16_t *fr = frame_ptr(m, f);
            double *pl = m->om[f];
#pragma omp parallel for schedule(static)
            for (int v = r0; v < r1; ++v)
                for (int u = 0; u < wh; ++u) {
                    double om[3];
                    omega_at(fr, m->h, m->w, u, v, m->p, m->wl, om);
                    for (int k = 0; k < 3; ++k) pl[k * rows * wh + (size_t)(v - r0) * wh + u] = om[k];
                }
        }
        if (f == m->ref) continue;
        /* Rhat rows (base grid) and the R rows they need (+-2) */
        int q0 = clampi((int)floor((ylo - 0.5) / 2.0) - 2, 0, hh);
        int q1 = clampi((int)ceil((yhi - 0.5) / 2.0) + 3, 0, hh);
        if (q1 <= q0) continue;
        int p0 = clampi(q0 - 2, 0, hh), p1 = clampi(q1 + 2, 0, hh);
        double *Rb = (double *)malloc(sizeof(double) * (size_t)(p1 - p0) * wh);
        m->rh[f] = (double *)malloc(sizeof(double) * (size_t)(q1 - q0) * wh);
        if (!Rb || !m->rh[f]) { free(Rb); return -2; }
        rob_geom g = { m->h, m->w, m->tile, m->ty, m->tx, m->wl, m->p };
        const uint16_t *base = frame_ptr(m, m->ref), *alt = frame_ptr(m, f);
        const float *mva = motion_ptr(m, f);
        const double *st = m->s_tile[f];
#pragma omp parallel for schedule(static)
        for (int v = p0; v < p1; ++v)
            for (int u = 0; u < wh; ++u) Rb[(size_t)(v - p0) * wh + u] = robustness_at(base, alt, mva, st, &g, u, v);
        double *rh = m->rh[f];
#pragma omp parallel for schedule(static)
        for (int v = q0; v < q1; ++v)
            for (int u = 0; u < wh; ++u) {
                double best = INFINITY;
                for (int j = -2; j <= 2; ++j)
                    for (int i = -2; i <= 2; ++i) {
                        int uu = u + i, vv = v + j;
                        if (uu < 0 || uu >= wh || vv < 0 || vv >= hh) continue;
                        double r = Rb[(size_t)(vv - p0) * wh + uu];
                        if (r < best) best = r;
                    }
                rh[(size_t)(v - q0) * wh + u] = best;
            }
        free(Rb);
        m->rh_r0[f] = q0; m->rh_r1[f] = q1;
    }
    return 0;
}

int orc_merge_rows(const uint16_t *burst, int n, int h, int w, int ref, const float *motion, int tile,
                   const orc_params *p, int wl, int snum, int sden, int y0, int y1, double *out,
                   double *den, int n_threads)
{
    if (snum < 1 || sden < 1 || !out) return -1;
    int ho = (int)(((long long)h * snum) / sden), wo = (int)(((long long)w * snum) / sden);
    if (y0 < 0 || y1 > ho || y1 < y0) return -1;
    set_threads(n_threads);
    merge_ctx m;
    int rc = init_ctx(&m, burst, n, h, w, ref, motion, tile, p, wl);
    if (rc == 0 && y1 > y0) rc = precompute_rows(&m, snum, sden, y0, y1);
    if (rc != 0) { free_ctx(&m); return rc; }
    size_t plane = (size_t)(y1 - y0) * wo;
#pragma omp parallel for schedule(dynamic, 1)
    for (int Y = y0; Y < y1; ++Y)
        for (int X = 0; X < wo; ++X) {
            double o[3], d[3];
            merge_pixel(&m, snum, sden, X, Y, o, d);
            size_t idx = (size_t)(Y - y0) * wo + X;
            for (int c = 0; c < 3; ++c) {
                out[c * plane + idx] = o[c];
                if (den) den[c * plane + idx] = d[c];
            }
        }
    free_ctx(&m);
    return 0;
}

int orc_merge_pixels(const uint16_t *burst, int n, int h, int w, int ref, const float *motion, int tile,
                     const orc_params *p, int wl, int snum, int sden, const int32_t *xy, int count,
                     double *out, int n_threads)
{
    if (snum < 1 || sden < 1 || !xy || !out || count < 0) return -1;
    int ho = (int)(((long long)h * snum) / sden), wo = (int)(((long long)w * snum) / sden);
    for (int k = 0; k < count; ++k)
        if (xy[2 * k] < 0 || xy[2 * k] >= wo || xy[2 * k + 1] < 0 || xy[2 * k + 1] >= ho) return -1;
    set_threads(n_threads);
    merge_ctx m;
    int rc = init_ctx(&m, burst, n, h, w, ref, motion, tile, p, wl);
    if (rc != 0) { free_ctx(&m); return rc; }
#pragma omp parallel for schedule(dynamic, 4)
    for (int k = 0; k < count; ++k) merge_pixel(&m, snum, sden, xy[2 * k], xy[2 * k + 1], out + 3 * (size_t)k, NULL);
    free_ctx(&m);
    return 0;
}

/* ------------------------------------------------------------------------------------ */
/* Alignment (Sec. 3.2): pyramid block matching, then Lucas-Kanade refinement            */
/* ------------------------------------------------------------------------------------ */
/* The paper follows Hasinoff et al.'s coarse-to-fine tile search without giving its
 * settings.  Readings taken: level 0 is Lq; level l+1 is the integer floor mean of
 * f x f blocks of level l with f = 2, 4, 4; tiles are tile/2 px at every level; a tile's
 * start vector is its parent's vector (the parent tile holds this tile's centre) times
 * f; the search covers offsets |dx|, |dy| <= radius[l]; the distance is the integer sum
 * of squared differences over the tile (reads clamped); ties go to the smallest SSD,
 * then the smallest |dx| + |dy|, then the smaller dy, then the smaller dx. */
typedef struct { int h, w; int32_t *px; } level_img;

static inline int32_t lvl_at(const level_img *L, int x, int y)
{
    x = clampi(x, 0, L->w - 1);
    y = clampi(y, 0, L->h - 1);
    return L->px[(size_t)y * L->w + x];
}

static const int kFactors[3] = { 2, 4, 4 };

static int build_pyramid(const uint16_t *raw, int h, int w, int n_levels_max, level_img *lv)
{
    int hh = h / 2, wh = w / 2;
    lv[0].h = hh; lv[0].w = wh;
    lv[0].px = (int32_t *)malloc(sizeof(int32_t) * (size_t)hh * wh);
    if (!lv[0].px) return -2;
    orc_luma(raw, h, w, lv[0].px);
    int nl = 1;
    while (nl < n_levels_max && nl < 4) {
        int f = kFactors[nl - 1];
        int nh = lv[nl - 1].h / f, nw = lv[nl - 1].w / f;
        if (nh < 16 || nw < 16) break;
        lv[nl].h = nh; lv[nl].w = nw;
        lv[nl].px = (int32_t *)malloc(sizeof(int32_t) * (size_t)nh * nw);
        if (!lv[nl].px) return -2;
        for (int y = 0; y < nh; ++y)
            for (int x = 0; x < nw; ++x) {
                int64_t s = 0;
                for (int j = 0; j < f; ++j)
                    for (int i = 0; i < f; ++i) s += lv[nl - 1].px[(size_t)(y * f + j) * lv[nl - 1].w + x * f + i];
                lv[nl].px[(size_t)y * nw + x] = (int32_t)(s / (f * f));
            }
        ++nl;
    }
    return nl;
}

/* One tile's integer search at one level: returns the best offset in (*bx, *by). */
static void tile_search(const level_img *Lr, const level_img *La, int t, int tx, int ty, int cx, int cy, int rad,
                        int *bx, int *by)
{
    int64_t best = -1;
    int bdx = 0, bdy = 0;
    for (int dy = -rad; dy <= rad; ++dy)
        for (int dx = -rad; dx <= rad; ++dx) {
            int64_t ssd = 0;
            for (int j = 0; j < t; ++j)
                for (int i = 0; i < t; ++i) {
                    int x = tx * t + i, y = ty * t + j;
                    int64_t d = (int64_t)lvl_at(Lr, x, y) - lvl_at(La, x + cx + dx, y + cy + dy);
                    ssd += d * d;
                }
            int better;
            if (best < 0 || ssd < best) better = 1;
            else if (ssd > best) better = 0;
            else {
                int m_new = abs(dx) + abs(dy), m_old = abs(bdx) + abs(bdy);
                if (m_new != m_old) better = m_new < m_old;
                else if (dy != bdy) better = dy < bdy;
                else better = dx < bdx;
            }
            if (better) { best = ssd; bdx = dx; bdy = dy; }
        }
    *bx = cx + bdx;
    *by = cy + bdy;
}

/* Lucas-Kanade refinement (three iterations in the paper) of one tile at level 0, on
 * I = Lq / 4.  Readings taken: gradients of the base frame by central differences
 * (clamped), H = sum g g^T over the tile, each iteration r(p) = I_alt(p + u + delta)
 * - I_ref(p) with bilinear sampling (clamped) and delta <- delta - H^-1 sum g r, delta
 * clamped to [-1, 1] per axis; the update is skipped when tr H == 0 or
 * det H <= 1e-9 tr(H)^2.  H is accumulated exactly in integers (64 H) and the guard is
 * evaluated exactly (128-bit integers), so any implementation takes the same decision. */
static int lk_tile(const level_img *Lr, const level_img *La, int t, int tx, int ty, int ux, int uy, int iters,
                   double *ox, double *oy)
{
    int64_t hxx = 0, hxy = 0, hyy = 0;
    for (int j = 0; j < t; ++j)
        for (int i = 0; i < t; ++i) {
            int x = clampi(tx * t + i, 0, Lr->w - 1), y = clampi(ty * t + j, 0, Lr->h - 1);
            int64_t gx = (int64_t)lvl_at(Lr, x + 1, y) - lvl_at(Lr, x - 1, y);
            int64_t gy = (int64_t)lvl_at(Lr, x, y + 1) - lvl_at(Lr, x, y - 1);
            hxx += gx * gx; hxy += gx * gy; hyy += gy * gy;
        }
    /* g = (Lq difference) / 8 since I = Lq / 4 and central differences halve */
    double Hxx = (double)hxx, Hxy = (double)hxy, Hyy = (double)hyy;
    /* guard evaluated exactly: 10^9 det H <= tr(H)^2 in 128-bit integers */
    __int128 det_i = (__int128)hxx * hyy - (__int128)hxy * hxy;
    __int128 tr_i = (__int128)hxx + hyy;
    double dx = 0.0, dy = 0.0;
    int skipped = (tr_i == 0) || ((__int128)1000000000 * det_i <= tr_i * tr_i);
    if (!skipped) {
        for (int it = 0; it < iters; ++it) {
            double bx = 0.0, by = 0.0;
            for (int j = 0; j < t; ++j)
                for (int i = 0; i < t; ++i) {
                    int x = clampi(tx * t + i, 0, Lr->w - 1), y = clampi(ty * t + j, 0, Lr->h - 1);
                    double gx = ((double)lvl_at(Lr, x + 1, y) - lvl_at(Lr, x - 1, y)) / 8.0;
                    double gy = ((double)lvl_at(Lr, x, y + 1) - lvl_at(Lr, x, y - 1)) / 8.0;
                    double sx = x + ux + dx, sy = y + uy + dy;
                    double fx0 = floor(sx), fy0 = floor(sy);
                    double ax = sx - fx0, ay = sy - fy0;
                    int ix = (int)fx0, iy = (int)fy0;
                    double i00 = lvl_at(La, ix, iy) / 4.0, i10 = lvl_at(La, ix + 1, iy) / 4.0;
                    double i01 = lvl_at(La, ix, iy + 1) / 4.0, i11 = lvl_at(La, ix + 1, iy + 1) / 4.0;
                    double ia = (1.0 - ay) * ((1.0 - ax) * i00 + ax * i10) + ay * ((1.0 - ax) * i01 + ax * i11);
                    double r = ia - lvl_at(Lr, x, y) / 4.0;
                    bx += gx * r;
                    by += gy * r;
                }
            /* H in units of the gradient g = diff / 8: H_g = H_int / 64 */
            double gxx = Hxx / 64.0, gxy = Hxy / 64.0, gyy = Hyy / 64.0;
            double gdet = gxx * gyy - gxy * gxy;
            double stepx = -(gyy * bx - gxy * by) / gdet;
            double stepy = -(-gxy * bx + gxx * by) / gdet;
            dx = clampd(dx + stepx, -1.0, 1.0);
            dy = clampd(dy + stepy, -1.0, 1.0);
        }
    }
    *ox = dx; *oy = dy;
    return skipped;
}

int orc_align(const uint16_t *burst, int n, int h, int w, int ref, int tile, int n_levels_max, const int *radius,
              int lk_iters, int32_t *motion_int, double *motion, int32_t *lk_flags, int n_threads)
{
    if (!burst || !radius || n < 1 || h < 4 || w < 4 || (h & 1) || (w & 1) || ref < 0 || ref >= n || tile < 2 ||
        (tile & 1) || n_levels_max < 1 || lk_iters < 0)
        return -1;
    set_threads(n_threads);
    int t = tile / 2;
    int ty0 = (h + tile - 1) / tile, tx0 = (w + tile - 1) / tile;
    level_img ref_lv[4];
    memset(ref_lv, 0, sizeof(ref_lv));
    int nl = build_pyramid(burst + (size_t)ref * h * w, h, w, n_levels_max, ref_lv);
    if (nl < 0) return nl;
    int rc = nl;
    for (int f = 0; f < n; ++f) {
        size_t off = (size_t)f * ty0 * tx0;
        if (f == ref) {
            for (size_t k = 0; k < (size_t)ty0 * tx0; ++k) {
                if (motion_int) { motion_int[2 * (off + k)] = 0; motion_int[2 * (off + k) + 1] = 0; }
                if (motion) { motion[2 * (off + k)] = 0.0; motion[2 * (off + k) + 1] = 0.0; }
                if (lk_flags) lk_flags[off + k] = 0;
            }
            continue;
        }
        level_img alt_lv[4];
        memset(alt_lv, 0, sizeof(alt_lv));
        int nla = build_pyramid(burst + (size_t)f * h * w, h, w, n_levels_max, alt_lv);
        if (nla != nl) { rc = -2; for (int l = 0; l < 4; ++l) free(alt_lv[l].px); break; }
        int *vec = NULL;   /* vectors of the previous (coarser) level */
        int pty = 0, ptx = 0;
        for (int l = nl - 1; l >= 0; --l) {
            int lty = (ref_lv[l].h + t - 1) / t, ltx = (ref_lv[l].w + t - 1) / t;
            int *cur = (int *)malloc(sizeof(int) * 2 * (size_t)lty * ltx);
            int fct = (l < nl - 1) ? kFactors[l] : 1;
#pragma omp parallel for schedule(static)
            for (int y = 0; y < lty; ++y)
                for (int x = 0; x < ltx; ++x) {
                    int cx = 0, cy = 0;
                    if (vec) {
                        int px = clampi((x * t + t / 2) / fct / t, 0, ptx - 1);
                        int py = clampi((y * t + t / 2) / fct / t, 0, pty - 1);
                        cx = vec[2 * ((size_t)py * ptx + px)] * fct;
                        cy = vec[2 * ((size_t)py * ptx + px) + 1] * fct;
                    }
                    int bx, by;
                    tile_search(&ref_lv[l], &alt_lv[l], t, x, y, cx, cy, radius[l], &bx, &by);
                    cur[2 * ((size_t)y * ltx + x)] = bx;
                    cur[2 * ((size_t)y * ltx + x) + 1] = by;
                }
            free(vec);
            vec = cur; pty = lty; ptx = ltx;
        }
        /* vec holds level-0 vectors on the ty0 x tx0 grid */
#pragma omp parallel for schedule(static)
        for (int y = 0; y < ty0; ++y)
            for (int x = 0; x < tx0; ++x) {
                size_t k = (size_t)y * tx0 + x;
                int ux = vec[2 * k], uy = vec[2 * k + 1];
                if (motion_int) { motion_int[2 * (off + k)] = ux; motion_int[2 * (off + k) + 1] = uy; }
                double ddx = 0.0, ddy = 0.0;
                int sk = lk_tile(&ref_lv[0], &alt_lv[0], t, x, y, ux, uy, lk_iters, &ddx, &ddy);
                if (lk_flags) lk_flags[off + k] = sk;
                if (motion) {
                    motion[2 * (off + k)] = 2.0 * (ux + ddx);
                    motion[2 * (off + k) + 1] = 2.0 * (uy + ddy);
                }
            }
        free(vec);
        for (int l = 0; l < 4; ++l) free(alt_lv[l].px);
    }
    for (int l = 0; l < 4; ++l) free(ref_lv[l].px);
    return rc;
}

/* ------------------------------------------------------------------------------------ */
/* Adjoint of the merge (reverse mode of Eq. 1-9 and the supplement's heuristics)        */
/* ------------------------------------------------------------------------------------ */
/* Differentiable parameters, in this order: k_detail, k_denoise, D_th, D_tr, k_stretch,
 * k_shrink, s (the robustness scale s2 of Eq. 8 used where the motion prior does not
 * fire; s1 stays fixed) and t.  Discrete decisions (window centres, tiles, s1/s2
 * selection, clamps, the 5x5 argmin, bilinear cells) carry no gradient: at such a point
 * the one-sided derivatives differ and the value used is that of the branch taken.
 *
 * Kernel shape derivative: d Omega / d p = (d k_across / d p) e1 e1^T + (d k_along / d p) e2 e2^T. */
static void kernel_param_grad(int64_t a, int64_t b, int64_t c, const orc_params *p, int wl, double dOm[6][3])
{
    double k[11];
    kernel_from_tensor(a, b, c, p, wl, k);
    double A = k[5], cs = k[9], sn = k[10];
    double l1 = k[3];
    double rl = sqrt(l1 / (4.0 * (8.0 * wl) * (8.0 * wl)));
    double Draw = 1.0 - rl / p->d_tr + p->d_th;
    double D = clampd(Draw, 0.0, 1.0);
    int inside = Draw > 0.0 && Draw < 1.0;
    double dD2 = inside ? 1.0 : 0.0, dD3 = inside ? rl / (p->d_tr * p->d_tr) : 0.0;
    double kh_al = p->k_detail * p->k_stretch * A, kh_ac = p->k_detail / (p->k_shrink * A);
    double kd = p->k_detail * p->k_denoise;
    double s_al = (1.0 - D) * kh_al + D * kd, s_ac = (1.0 - D) * kh_ac + D * kd;
    double ds_al[6] = { (1.0 - D) * p->k_stretch * A + D * p->k_denoise, D * p->k_detail,
                        (kd - kh_al) * dD2, (kd - kh_al) * dD3, (1.0 - D) * p->k_detail * A, 0.0 };
    double ds_ac[6] = { (1.0 - D) / (p->k_shrink * A) + D * p->k_denoise, D * p->k_detail,
                        (kd - kh_ac) * dD2, (kd - kh_ac) * dD3, 0.0,
                        -(1.0 - D) * p->k_detail / (p->k_shrink * p->k_shrink * A) };
    double e1xx = 0.5 * (1.0 + cs), e1xy = 0.5 * sn, e1yy = 0.5 * (1.0 - cs);
    for (int q = 0; q < 6; ++q) {
        double dal = 2.0 * s_al * ds_al[q], dac = 2.0 * s_ac * ds_ac[q];
        dOm[q][0] = dac * e1xx + dal * (1.0 - e1xx);
        dOm[q][1] = dac * e1xy - dal * e1xy;
        dOm[q][2] = dac * e1yy + dal * (1.0 - e1yy);
    }
}

/* Robustness R at base half-res (u,v) for frame `alt` with its partial derivatives:
 * dR[0] = dR/dvx, dR[1] = dR/dvy (the tile's vector), dR[2] = dR/ds2, dR[3] = dR/dt.
 * Same arithmetic as robustness_at. */
static double robustness_grad_at(const uint16_t *base, const uint16_t *alt, const float *motion_alt,
                                 const double *s_tile, const rob_geom *g, int u, int v, double dR[4])
{
    const orc_params *p = g->p;
    int tyi = clampi((2 * v) / g->tile, 0, g->ty - 1);
    int txi = clampi((2 * u) / g->tile, 0, g->tx - 1);
    const float *mv = motion_alt + ((size_t)tyi * g->tx + txi) * 2;
    double fx = (double)u + 0.5 * (double)mv[0];
    double fy = (double)v + 0.5 * (double)mv[1];
    double x0 = floor(fx), y0 = floor(fy);
    double ax = fx - x0, ay = fy - y0;
    int ix = (int)x0, iy = (int)y0;
    double dd = 0.0, ss = 0.0, ddd_dvx = 0.0, ddd_dvy = 0.0;
    for (int c = 0; c < 3; ++c) {
        double s1 = (double)box_sum(base, g->h, g->w, u, v, c, 0);
        double s2 = (double)box_sum(base, g->h, g->w, u, v, c, 1);
        double gs = (c == 1) ? 2.0 : 1.0;
        double mu = s1 / (9.0 * gs);
        double var_ms = (9.0 * s2 - s1 * s1) / (81.0 * gs * gs);
        if (var_ms < 0.0) var_ms = 0.0;
        double sigma_ms = sqrt(var_ms);
        double m00 = box_mean(alt, g->h, g->w, ix, iy, c), m10 = box_mean(alt, g->h, g->w, ix + 1, iy, c);
        double m01 = box_mean(alt, g->h, g->w, ix, iy + 1, c), m11 = box_mean(alt, g->h, g->w, ix + 1, iy + 1, c);
        double mu_n = (1.0 - ay) * ((1.0 - ax) * m00 + ax * m10) + ay * ((1.0 - ax) * m01 + ax * m11);
        double dmu_dfx = (1.0 - ay) * (m10 - m00) + ay * (m11 - m01);
        double dmu_dfy = (1.0 - ax) * (m01 - m00) + ax * (m11 - m10);
        double d_ms = mu - mu_n;
        double var_md, m;
        modelled_stats(p, g->wl, mu, c, &var_md, &m);
        double sigma_md = sqrt(var_md);
        double sigma = sigma_ms > sigma_md ? sigma_ms : sigma_md;
        double den = d_ms * d_ms + m;
        double d = den > 0.0 ? d_ms * (d_ms * d_ms) / den : 0.0;
        double dd_dms = den > 0.0 ? (d_ms * d_ms * d_ms * d_ms + 3.0 * m * d_ms * d_ms) / (den * den) : 0.0;
        dd += d * d;
        ss += sigma * sigma;
        /* d(d^2)/d v = 2 d dd/dd_ms * (-dmu_n/dpos) * 1/2 */
        ddd_dvx += 2.0 * d * dd_dms * (-dmu_dfx) * 0.5;
        ddd_dvy += 2.0 * d * dd_dms * (-dmu_dfy) * 0.5;
    }
    double eps = 1e-12 * (double)g->wl * (double)g->wl;
    double S = ss > eps ? ss : eps;
    double ratio = dd / S;
    double s = s_tile[(size_t)tyi * g->tx + txi];
    double e = exp(-ratio);
    double raw = s * e - p->t;
    double R = clampd(raw, 0.0, 1.0);
    if (raw > 0.0 && raw < 1.0) {
        dR[0] = -s * e * ddd_dvx / S;
        dR[1] = -s * e * ddd_dvy / S;
        dR[2] = (tile_M(motion_alt, g->ty, g->tx, tyi, txi) > p->m_th) ? 0.0 : e;   /* s = s2 here */
        dR[3] = -1.0;
    } else {
        dR[0] = dR[1] = dR[2] = dR[3] = 0.0;
    }
    return R;
}

int orc_merge_backward(const uint16_t *burst, int n, int h, int w, int ref, const float *motion, int tile,
                       const orc_params *p, int wl, int snum, int sden, const double *grad_out,
                       double *grad_params, double *grad_motion, int n_threads)
{
    if (!grad_out || !grad_params || !grad_motion || snum < 1 || sden < 1) return -1;
    set_threads(n_threads);
    merge_ctx m;
    int rc = init_ctx(&m, burst, n, h, w, ref, motion, tile, p, wl);
    int ho = (int)(((long long)h * snum) / sden), wo = (int)(((long long)w * snum) / sden);
    if (rc == 0) rc = precompute_rows(&m, snum, sden, 0, ho);
    if (rc != 0) { free_ctx(&m); return rc; }
    const int hh = h / 2, wh = w / 2;
    const size_t hw = (size_t)hh * wh;
    rob_geom g = { h, w, tile, m.ty, m.tx, wl, p };
    /* per-frame accumulators: Omega-bar per texel, Rhat-bar per base texel */
    double *om_bar = (double *)calloc((size_t)n * 3 * hw, sizeof(double));
    double *rh_bar = (double *)calloc((size_t)n * hw, sizeof(double));
    memset(grad_params, 0, 8 * sizeof(double));
    memset(grad_motion, 0, sizeof(double) * (size_t)n * m.ty * m.tx * 2);
    if (!om_bar || !rh_bar) { free(om_bar); free(rh_bar); free_ctx(&m); return -2; }
    const long long Q = 2LL * snum;
    for (int Y = 0; Y < ho; ++Y)
        for (int X = 0; X < wo; ++X) {
            double C[3], den[3];
            merge_pixel(&m, snum, sden, X, Y, C, den);
            const long long Px = 2LL * sden * X + sden - snum, Py = 2LL * sden * Y + sden - snum;
            const double x0 = (double)Px / (double)Q, y0 = (double)Py / (double)Q;
            int txi = clampi((int)floor_div(Px, Q * tile), 0, m.tx - 1);
            int tyi = clampi((int)floor_div(Py, Q * tile), 0, m.ty - 1);
            double gc[3];
            for (int c = 0; c < 3; ++c) gc[c] = grad_out[(size_t)c * ho * wo + (size_t)Y * wo + X];
            for (int f = 0; f < n; ++f) {
                double vx = 0.0, vy = 0.0;
                if (f != ref) {
                    const float *mv = motion_ptr(&m, f) + ((size_t)tyi * m.tx + txi) * 2;
                    vx = (double)mv[0];
                    vy = (double)mv[1];
                }
                long long kx = floor_div(Px + Q / 2 + (long long)floor((double)Q * vx), Q);
                long long ky = floor_div(Py + Q / 2 + (long long)floor((double)Q * vy), Q);
                double px = x0 + vx, py = y0 + vy;
                double hx = (px - 0.5) / 2.0, hy = (py - 0.5) / 2.0;
                double fx0 = floor(hx), fy0 = floor(hy);
                double ax = hx - fx0, ay = hy - fy0;
                int ix = (int)fx0, iy = (int)fy0;
                int tx_[4] = { clampi(ix, 0, wh - 1), clampi(ix + 1, 0, wh - 1), clampi(ix, 0, wh - 1), clampi(ix + 1, 0, wh - 1) };
                int ty_[4] = { clampi(iy, 0, hh - 1), clampi(iy, 0, hh - 1), clampi(iy + 1, 0, hh - 1), clampi(iy + 1, 0, hh - 1) };
                double beta[4] = { (1 - ax) * (1 - ay), ax * (1 - ay), (1 - ax) * ay, ax * ay };
                double dbx[4] = { -(1 - ay), (1 - ay), -ay, ay };     /* d beta / d ax */
                double dby[4] = { -(1 - ax), -ax, (1 - ax), ax };     /* d beta / d ay */
                double ok[4][3], om[3] = { 0, 0, 0 };
                for (int k = 0; k < 4; ++k) {
                    omega_get(&m, f, tx_[k], ty_[k], ok[k]);
                    for (int e = 0; e < 3; ++e) om[e] += beta[k] * ok[k][e];
                }
                double det = om[0] * om[2] - om[1] * om[1];
                double ixx = om[2] / det, ixy = -om[1] / det, iyy = om[0] / det;
                double rhat = 1.0, gam[4] = { 0, 0, 0, 0 };
                int gx_[4] = { 0, 0, 0, 0 }, gy_[4] = { 0, 0, 0, 0 };
                if (f != ref) {
                    double gx = (x0 - 0.5) / 2.0, gy = (y0 - 0.5) / 2.0;
                    double gx0 = floor(gx), gy0 = floor(gy);
                    double bx = gx - gx0, by = gy - gy0;
                    int jx = (int)gx0, jy = (int)gy0;
                    gx_[0] = clampi(jx, 0, wh - 1); gx_[1] = clampi(jx + 1, 0, wh - 1); gx_[2] = gx_[0]; gx_[3] = gx_[1];
                    gy_[0] = clampi(jy, 0, hh - 1); gy_[1] = gy_[0]; gy_[2] = clampi(jy + 1, 0, hh - 1); gy_[3] = gy_[2];
                    gam[0] = (1 - bx) * (1 - by); gam[1] = bx * (1 - by); gam[2] = (1 - bx) * by; gam[3] = bx * by;
                    rhat = 0.0;
                    for (int k = 0; k < 4; ++k) rhat += gam[k] * rhat_get(&m, f, gx_[k], gy_[k]);
                }
                const uint16_t *fr = frame_ptr(&m, f);
                double om_b[3] = { 0, 0, 0 }, v_b[2] = { 0, 0 }, rh_b = 0.0;
                for (int j = -1; j <= 1; ++j)
                    for (int i = -1; i <= 1; ++i) {
                        long long qx = kx + i, qy = ky + j;
                        if (qx < 0 || qx >= w || qy < 0 || qy >= h) continue;
                        double dx = (double)qx - px, dy = (double)qy - py;
                        double Pxv = ixx * dx + ixy * dy, Pyv = ixy * dx + iyy * dy;   /* Omega^-1 d */
                        double qf = dx * Pxv + dy * Pyv;
                        double wgt = exp(-0.5 * qf);
                        int c = cfa_channel((int)qx, (int)qy);
                        double cval = (double)fr[(size_t)qy * w + qx];
                        double gwr = gc[c] * (cval - C[c]) / den[c];   /* dL / d(w Rhat) */
                        rh_b += gwr * wgt;
                        double q_b = gwr * rhat * (-0.5 * wgt);           /* dL / dq */
                        /* q = d^T Omega^-1 d: dq/dd = 2 Omega^-1 d, dq/dv = -dq/dd */
                        v_b[0] += -2.0 * q_b * Pxv;
                        v_b[1] += -2.0 * q_b * Pyv;
                        /* dq/dOmega = -(Omega^-1 d)(Omega^-1 d)^T; Oxy counted twice */
                        om_b[0] += -q_b * Pxv * Pxv;
                        om_b[1] += -2.0 * q_b * Pxv * Pyv;
                        om_b[2] += -q_b * Pyv * Pyv;
                    }
                /* Omega position: h = (x0 + v - 1/2)/2, so d(ax)/d(vx) = 1/2 */
                for (int k = 0; k < 4; ++k) {
                    double dot = om_b[0] * ok[k][0] + om_b[1] * ok[k][1] + om_b[2] * ok[k][2];
                    v_b[0] += 0.5 * dbx[k] * dot;
                    v_b[1] += 0.5 * dby[k] * dot;
                    for (int e = 0; e < 3; ++e)
                        om_bar[((size_t)f * 3 + e) * hw + (size_t)ty_[k] * wh + tx_[k]] += beta[k] * om_b[e];
                }
                if (f != ref) {
                    double *gm = grad_motion + ((size_t)f * m.ty * m.tx + (size_t)tyi * m.tx + txi) * 2;
                    gm[0] += v_b[0];
                    gm[1] += v_b[1];
                    for (int k = 0; k < 4; ++k) rh_bar[(size_t)f * hw + (size_t)gy_[k] * wh + gx_[k]] += gam[k] * rh_b;
                }
            }
        }
    /* texels: Omega-bar -> kernel parameters */
    for (int f = 0; f < n; ++f)
        for (int v = 0; v < hh; ++v)
            for (int u = 0; u < wh; ++u) {
                double ob[3];
                for (int e = 0; e < 3; ++e) ob[e] = om_bar[((size_t)f * 3 + e) * hw + (size_t)v * wh + u];
                if (ob[0] == 0.0 && ob[1] == 0.0 && ob[2] == 0.0) continue;
                int64_t a, b, c;
                tensor_at(frame_ptr(&m, f), h, w, u, v, &a, &b, &c);
                double dOm[6][3];
                kernel_param_grad(a, b, c, p, wl, dOm);
                for (int q = 0; q < 6; ++q) grad_params[q] += ob[0] * dOm[q][0] + ob[1] * dOm[q][1] + ob[2] * dOm[q][2];
            }
    /* Rhat-bar -> argmin R -> s, t and the motion of the R pixel's tile */
    double *Rpl = (double *)malloc(sizeof(double) * hw);
    double *dRpl = (double *)malloc(sizeof(double) * hw * 4);
    double *Rbar = (double *)malloc(sizeof(double) * hw);
    if (!Rpl || !dRpl || !Rbar) { free(Rpl); free(dRpl); free(Rbar); free(om_bar); free(rh_bar); free_ctx(&m); return -2; }
    for (int f = 0; f < n; ++f) {
        if (f == ref) continue;
        const uint16_t *base = frame_ptr(&m, ref), *alt = frame_ptr(&m, f);
        for (int v = 0; v < hh; ++v)
            for (int u = 0; u < wh; ++u)
                Rpl[(size_t)v * wh + u] = robustness_grad_at(base, alt, motion_ptr(&m, f), m.s_tile[f], &g, u, v,
                                                             &dRpl[((size_t)v * wh + u) * 4]);
        memset(Rbar, 0, sizeof(double) * hw);
        for (int v = 0; v < hh; ++v)
            for (int u = 0; u < wh; ++u) {
                double rb = rh_bar[(size_t)f * hw + (size_t)v * wh + u];
                if (rb == 0.0) continue;
                /* first minimum of the 5x5 window in scan order */
                double best = INFINITY;
                int bu = u, bv = v;
                for (int j = -2; j <= 2; ++j)
                    for (int i = -2; i <= 2; ++i) {
                        int uu = u + i, vv = v + j;
                        if (uu < 0 || uu >= wh || vv < 0 || vv >= hh) continue;
                        double r = Rpl[(size_t)vv * wh + uu];
                        if (r < best) { best = r; bu = uu; bv = vv; }
                    }
                Rbar[(size_t)bv * wh + bu] += rb;
            }
        const float *mva = motion_ptr(&m, f);
        (void)mva;
        for (int v = 0; v < hh; ++v)
            for (int u = 0; u < wh; ++u) {
                double rb = Rbar[(size_t)v * wh + u];
                if (rb == 0.0) continue;
                const double *dR = &dRpl[((size_t)v * wh + u) * 4];
                int tyi = clampi((2 * v) / tile, 0, m.ty - 1), txi = clampi((2 * u) / tile, 0, m.tx - 1);
                double *gm = grad_motion + ((size_t)f * m.ty * m.tx + (size_t)tyi * m.tx + txi) * 2;
                gm[0] += rb * dR[0];
                gm[1] += rb * dR[1];
                grad_params[6] += rb * dR[2];
                grad_params[7] += rb * dR[3];
            }
    }
    free(Rpl); free(dRpl); free(Rbar); free(om_bar); free(rh_bar);
    free_ctx(&m);
    return 0;
}

/* A fingerprint of every discrete decision of the merge at these arguments (window
 * centres, motion-prior selections, clamp states of D and R, 5x5 argmins).  Finite
 * differences are only meaningful between points with equal fingerprints. */
unsigned long long orc_merge_fingerprint(const uint16_t *burst, int n, int h, int w, int ref, const float *motion,
                                         int tile, const orc_params *p, int wl, int snum, int sden)
{
    merge_ctx m;
    if (init_ctx(&m, burst, n, h, w, ref, motion, tile, p, wl) != 0) { free_ctx(&m); return 0; }
    unsigned long long hsh = 1469598103934665603ULL;
#define MIX(x) do { hsh ^= (unsigned long long)(x); hsh *= 1099511628211ULL; } while (0)
    int ho = (int)(((long long)h * snum) / sden), wo = (int)(((long long)w * snum) / sden);
    const long long Q = 2LL * snum;
    const int hh = h / 2, wh = w / 2;
    for (int Y = 0; Y < ho; ++Y)
        for (int X = 0; X < wo; ++X) {
            const long long Px = 2LL * sden * X + sden - snum, Py = 2LL * sden * Y + sden - snum;
            int txi = clampi((int)floor_div(Px, Q * tile), 0, m.tx - 1);
            int tyi = clampi((int)floor_div(Py, Q * tile), 0, m.ty - 1);
            for (int f = 0; f < n; ++f) {
                double vx = 0.0, vy = 0.0;
                if (f != ref) {
                    const float *mv = motion_ptr(&m, f) + ((size_t)tyi * m.tx + txi) * 2;
                    vx = mv[0]; vy = mv[1];
                }
                MIX(floor_div(Px + Q / 2 + (long long)floor((double)Q * vx), Q));
                MIX(floor_div(Py + Q / 2 + (long long)floor((double)Q * vy), Q));
                MIX((long long)floor(((double)Px / Q + vx - 0.5) / 2.0));
                MIX((long long)floor(((double)Py / Q + vy - 0.5) / 2.0));
            }
        }
    rob_geom g = { h, w, tile, m.ty, m.tx, wl, p };
    double *Rpl = (double *)malloc(sizeof(double) * (size_t)hh * wh);
    for (int f = 0; f < n && Rpl; ++f) {
        for (int v = 0; v < hh; ++v)
            for (int u = 0; u < wh; ++u) {
                int64_t a, b, c;
                double k[11];
                tensor_at(frame_ptr(&m, f), h, w, u, v, &a, &b, &c);
                kernel_from_tensor(a, b, c, p, wl, k);
                double rl = sqrt(k[3] / (4.0 * (8.0 * wl) * (8.0 * wl)));
                double Draw = 1.0 - rl / p->d_tr + p->d_th;
                MIX(Draw <= 0.0 ? 0 : (Draw >= 1.0 ? 2 : 1));
            }
        if (f == ref) continue;
        for (int t = 0; t < m.ty * m.tx; ++t) MIX(m.s_tile[f][t] == p->s1);
        for (int v = 0; v < hh; ++v)
            for (int u = 0; u < wh; ++u) {
                double dR[4];
                Rpl[(size_t)v * wh + u] = robustness_grad_at(frame_ptr(&m, ref), frame_ptr(&m, f), motion_ptr(&m, f),
                                                             m.s_tile[f], &g, u, v, dR);
                MIX(dR[3] != 0.0);
                int tyi = clampi((2 * v) / tile, 0, m.ty - 1), txi = clampi((2 * u) / tile, 0, m.tx - 1);
                const float *mv = motion_ptr(&m, f) + ((size_t)tyi * m.tx + txi) * 2;
                MIX((long long)floor(u + 0.5 * mv[0]));
                MIX((long long)floor(v + 0.5 * mv[1]));
            }
        for (int v = 0; v < hh; ++v)
            for (int u = 0; u < wh; ++u) {
                double best = INFINITY;
                int bi = 0;
                for (int j = -2; j <= 2; ++j)
                    for (int i = -2; i <= 2; ++i) {
                        int uu = u + i, vv = v + j;
                        if (uu < 0 || uu >= wh || vv < 0 || vv >= hh) continue;
                        double r = Rpl[(size_t)vv * wh + uu];
                        if (r < best) { best = r; bi = (j + 2) * 5 + i + 2; }
                    }
                MIX(bi);
            }
    }
#undef MIX
    free(Rpl);
    free_ctx(&m);
    return hsh;
}


/* ======================================================================================
 * Monte-Carlo noise statistics (Sec. 5.2.2)
 * ==================================================================================== */
void orc_philox(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    /* Philox-4x32 with 10 rounds: per round two 32x32 -> 64-bit products by the fixed
     * multipliers, the halves recombined with the other counter words and the round key,
     * the key bumped by the Weyl constants between rounds */
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3], k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t p0 = (uint64_t)0xD2511F53u * c0, p1 = (uint64_t)0xCD9E8D57u * c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0, hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
        c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* the j-th normal of trial `trial` at level `level`: 12 uniforms (r + 1/2) 2^-32 from
 * three Philox blocks, summed exactly, minus 6 */
static double noise_normal(int level, int trial, int j)
{
    static const uint32_t key[2] = {0x19050327u, 0x5EED0001u};
    uint64_t s = 0;
    for (int b = 0; b < 3; ++b) {
        uint32_t ctr[4] = {(uint32_t)(3 * j + b), (uint32_t)trial, (uint32_t)level, 0u}, out[4];
        orc_philox(ctr, key, out);
        s += (uint64_t)out[0] + out[1] + out[2] + out[3];
    }
    return ((double)s + 6.0) * (1.0 / 4294967296.0) - 6.0;
}

static double noise_sample(double x, double sigma, int wl, int level, int trial, int j)
{
    double v = floor(x + sigma * noise_normal(level, trial, j) + 0.5);
    return clampd(v, 0.0, (double)wl);
}

void orc_noise_table(double noise_a, double noise_b, int wl, double *table)
{
#pragma omp parallel for schedule(dynamic)
    for (int i = 0; i < ORC_NOISE_LEVELS; ++i) {
        double x = (double)i * (double)wl / (double)(ORC_NOISE_LEVELS - 1);
        double var = noise_a * x + noise_b;
        double sigma = var > 0.0 ? sqrt(var) : 0.0;
        double acc[4] = {0.0, 0.0, 0.0, 0.0};
        for (int t = 0; t < ORC_NOISE_TRIALS; ++t) {
            /* normals 0..8: patch 1 red/blue; 9..26: patch 1 green pairs;
             * 27..35: patch 2 red/blue; 36..53: patch 2 green pairs */
            double rb[2][9], gr[2][9];
            for (int q = 0; q < 2; ++q)
                for (int k = 0; k < 9; ++k) {
                    rb[q][k] = noise_sample(x, sigma, wl, i, t, 27 * q + k);
                    gr[q][k] = 0.5 * (noise_sample(x, sigma, wl, i, t, 27 * q + 9 + 2 * k) +
                                      noise_sample(x, sigma, wl, i, t, 27 * q + 10 + 2 * k));
                }
            double mean[2][2], var1[2];
            for (int ch = 0; ch < 2; ++ch) {
                for (int q = 0; q < 2; ++q) {
                    double s = 0.0;
                    for (int k = 0; k < 9; ++k) s += ch ? gr[q][k] : rb[q][k];
                    mean[ch][q] = s / 9.0;
                }
                double ss = 0.0;
                for (int k = 0; k < 9; ++k) {
                    double d = (ch ? gr[0][k] : rb[0][k]) - mean[ch][0];
                    ss += d * d;
                }
                var1[ch] = ss / 9.0;
            }
            acc[0] += var1[0];
            acc[1] += var1[1];
            acc[2] += (mean[0][0] - mean[0][1]) * (mean[0][0] - mean[0][1]);
            acc[3] += (mean[1][0] - mean[1][1]) * (mean[1][0] - mean[1][1]);
        }
        for (int k = 0; k < 4; ++k) table[4 * i + k] = acc[k] / (double)ORC_NOISE_TRIALS;
    }
}
