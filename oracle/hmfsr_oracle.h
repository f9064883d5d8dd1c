/*
 * FP64 reference ("oracle") for the handheld multi-frame super-resolution merge and its
 * tile alignment (Wronski et al., "Handheld Multi-Frame Super-Resolution", 2019).
 *
 * TEST INFRASTRUCTURE ONLY.  This library is a plain, slow, obviously-correct CPU
 * restatement of the method, used to check the CUDA path.  Only the tests, the smoke
 * check and the benchmark's CPU-baseline leg may load it.  It shares no code, header,
 * table or helper with the CUDA path.
 *
 * Conventions (all host pointers, row-major, caller-owned):
 *   burst    uint16 [n][h][w], RGGB Bayer, (even x, even y) = R, (odd, odd) = B.
 *   half-res (u, v) covers raw (2u..2u+1, 2v..2v+1); hh = h/2, wh = w/2.
 *   motion   float32 [n][ty][tx][2] (x, y), base -> frame displacement in raw px,
 *            one vector per tile of `tile` raw px; ty = ceil(h/tile), tx = ceil(w/tile).
 *   output   double [3][ho][wo] (R, G, B) in DN.
 * Return value: 0 on success, negative on invalid arguments.
 */
#ifndef HMFSR_ORACLE_H
#define HMFSR_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Merge tuning parameters (supplement S.1 / S.2 and Sec. 5.2).  The values are the
 * float32 numbers the caller uses, promoted to double. */
typedef struct {
    double k_detail, k_denoise, d_th, d_tr, k_stretch, k_shrink;
    double t, s1, s2, m_th;
    double noise_a, noise_b;   /* noise variance = noise_a * x + noise_b (DN^2) */
    /* NULL: the closed-form noise statistics; else ORC_NOISE_LEVELS x 4 values from
     * orc_noise_table (Monte-Carlo sigma_md^2 and d_md^2 per brightness level) */
    const double *noise_table;
    /* 0: off; else the high-frequency rejection threshold kappa (supplement, High
     * Frequency Artifacts Removal): R = 0 where the variance of the 3x3 local means is
     * below kappa times the local variance and the tile's motion span M exceeds m_th */
    double hf_loss;
} orc_params;

/* Monte-Carlo noise statistics (Sec. 5.2.2: sigma_md and d_md "through a series of Monte
 * Carlo simulations for different brightness levels", with sensor clipping).  Level i of
 * ORC_NOISE_LEVELS is brightness x_i = i WL / (ORC_NOISE_LEVELS - 1).  Each of
 * ORC_NOISE_TRIALS trials draws two independent constant patches of 3x3 guide pixels:
 * red/blue guide = one raw sample, green guide = the mean of two; a raw sample is
 * clamp(floor(x + sqrt(a x + b) z + 1/2), 0, WL) with z an Irwin-Hall normal (sum of 12
 * uniforms - 6) from Philox-4x32-10.  Per level, table[4 i ..] = the trial means of
 * {population variance of patch 1, red/blue; the same, green; (mean of patch 1 - mean of
 * patch 2)^2, red/blue; the same, green}. */
#define ORC_NOISE_LEVELS 129
#define ORC_NOISE_TRIALS 4096
void orc_noise_table(double noise_a, double noise_b, int wl, double *table);

/* Philox-4x32-10 (Salmon et al., SC 2011) of counter ctr[4] under key[2] into out[4]. */
void orc_philox(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);

/* Half-res luminance Lq(u,v) = sum of the 4 Bayer samples of quad (u,v) (Sec. 5.1.2). */
int orc_luma(const uint16_t *raw, int h, int w, int32_t *lq);

/* Integer structure tensor (a, b, c) = (sum gx^2, sum gx gy, sum gy^2) at (u,v) (Eq. 3). */
int orc_structure_tensor(const uint16_t *raw, int h, int w, int u, int v, int64_t out[3]);

/* Kernel shape from a tensor (Eq. 4 and the supplement's heuristics S.1).
 * out = {Oxx, Oxy, Oyy, lambda1, lambda2, A, D, k_along, k_across, cos2t, sin2t}. */
int orc_kernel_from_tensor(int64_t a, int64_t b, int64_t c, const orc_params *p, int wl,
                           double out[11]);

/* Omega planes [3][hh][wh] of one frame. */
int orc_omega_plane(const uint16_t *raw, int h, int w, const orc_params *p, int wl, double *omega);

/* Motion strength M (Eq. 7) and the robustness scale s (Eq. 8) of each tile of one
 * frame's motion field [ty][tx][2].  M, s: double [ty][tx] (either may be NULL). */
int orc_tile_strength(const float *motion, int ty, int tx, const orc_params *p, double *M, double *s);

/* Robustness of frame `alt` against the base frame on the base half-res grid:
 * R (Eq. 5-6, clamped to [0,1]) and Rhat = 5x5 min of R (Eq. 9).  Either may be NULL. */
int orc_robustness(const uint16_t *base, const uint16_t *alt, int h, int w,
                   const float *motion_alt, int tile, const orc_params *p, int wl,
                   double *R, double *Rhat);

/* Merge (Eq. 1-2) of output rows [y0, y1) at scale snum/sden.
 * out: double [3][y1-y0][wo]; den (nullable): double [3][y1-y0][wo] = sum of w * Rhat. */
int orc_merge_rows(const uint16_t *burst, int n, int h, int w, int ref, const float *motion,
                   int tile, const orc_params *p, int wl, int snum, int sden, int y0, int y1,
                   double *out, double *den, int n_threads);

/* Merge of a list of output pixels xy[count][2] = (X, Y).  out: double [count][3]. */
int orc_merge_pixels(const uint16_t *burst, int n, int h, int w, int ref, const float *motion,
                     int tile, const orc_params *p, int wl, int snum, int sden,
                     const int32_t *xy, int count, double *out, int n_threads);

/* Tile alignment (Sec. 3.2).  Pyramid levels from Lq with factors 2, 4, 4 (integer floor
 * mean), a level is added while both of its sides are >= 16 px, at most n_levels_max
 * levels (<= 4).  radius[l] is the search radius at level l (0 = finest).  Tiles are
 * tile/2 level px at every level.
 * motion_int (nullable): int32 [n][ty][tx][2], integer vectors in half-res px.
 * motion:                double [n][ty][tx][2], after lk_iters Lucas-Kanade steps, raw px.
 * lk_flags (nullable):   int32 [n][ty][tx], 1 if the LK update was skipped (ill-conditioned).
 * Returns the number of levels used (> 0) or a negative error. */
int orc_align(const uint16_t *burst, int n, int h, int w, int ref, int tile, int n_levels_max,
              const int *radius, int lk_iters, int32_t *motion_int, double *motion,
              int32_t *lk_flags, int n_threads);

/* Adjoint of the merge: given dL/dC (double [3][ho][wo]) returns dL/dparams (double [8]:
 * k_detail, k_denoise, d_th, d_tr, k_stretch, k_shrink, s2, t) and dL/dmotion (double
 * [n][ty][tx][2]; zero for the base frame). */
int orc_merge_backward(const uint16_t *burst, int n, int h, int w, int ref, const float *motion, int tile,
                       const orc_params *p, int wl, int snum, int sden, const double *grad_out,
                       double *grad_params, double *grad_motion, int n_threads);

/* Fingerprint of the discrete decisions of the merge (for finite-difference checks). */
unsigned long long orc_merge_fingerprint(const uint16_t *burst, int n, int h, int w, int ref, const float *motion,
                                         int tile, const orc_params *p, int wl, int snum, int sden);

#ifdef __cplusplus
}
#endif
#endif
