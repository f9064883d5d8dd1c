/*
 * hmfsr — handheld multi-frame super-resolution (Wronski et al., "Handheld Multi-Frame
 * Super-Resolution", ACM TOG 38(4), 2019) on one GPU (sm_103a).
 *
 * C ABI.  Every call takes plain pointers and sizes.  Device pointers are CUDA device
 * memory owned by the caller; the library never allocates device memory on these calls:
 * scratch space is the caller's `ws` buffer, whose size is queried first with
 * hmfsr_workspace_size().  `stream` is a cudaStream_t passed as void* (NULL = legacy
 * default stream).  Calls are asynchronous on `stream`: arguments are validated on the
 * host before any launch (errors return without touching the GPU); a failed launch
 * returns HMFSR_ERR_CUDA.  The first merge call on a device also queries two kernels'
 * occupancy (host-side, once; no allocation, no synchronisation) to choose launch
 * shapes; results never depend on them.
 *
 * Image conventions (all calls):
 *   raw frames  uint16, RGGB Bayer: pixel (x, y) is R when x, y are both even, B when both
 *               odd, G otherwise.  Frame f, row y, column x is at
 *               burst[(f * height + y) * pitch_elems + x].  Values 0..white_level.
 *   half-res    pixel (u, v) covers raw (2u..2u+1, 2v..2v+1); its centre is raw
 *               (2u + 1/2, 2v + 1/2).
 *   tiles       square, `tile` raw px (even); tile (tx, ty) covers raw
 *               [tile*tx, tile*tx + tile) x [tile*ty, tile*ty + tile);
 *               TX = ceil(width / tile), TY = ceil(height / tile).
 *   motion      float32 [n_frames][TY][TX][2] = (vx, vy): the base -> frame displacement
 *               of each tile in raw px (a scene point at base position p is seen at
 *               p + v in that frame).  The base frame's entry is ignored (taken as 0).
 *   output      float32 planar [3][Ho][Wo] (R, G, B) in DN, Ho = floor(height*num/den),
 *               Wo = floor(width*num/den); output pixel X sits at raw (X + 1/2)*den/num - 1/2.
 */
#ifndef HMFSR_H
#define HMFSR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    HMFSR_OK = 0,
    HMFSR_ERR_INVALID_ARG = -1,  /* a pointer, size, stride or parameter is out of range */
    HMFSR_ERR_UNSUPPORTED = -2,  /* valid but not implemented (e.g. a non-RGGB CFA)      */
    HMFSR_ERR_WORKSPACE = -3,    /* ws is NULL, misaligned or smaller than required       */
    HMFSR_ERR_CUDA = -4,         /* a CUDA launch or runtime call failed                   */
    HMFSR_ERR_TIMEOUT = -5       /* a bounded device-side wait gave up                     */
} hmfsr_status;

/* One burst in device memory (Sec. 3.1: a burst of raw CFA frames and a base frame). */
typedef struct {
    int n_frames;      /* >= 1                                                   */
    int height, width; /* raw frame size, both even, >= 4                          */
    int pitch_elems;   /* row stride in elements, even, >= width                   */
    int ref;           /* index of the base frame, 0 <= ref < n_frames             */
    int cfa;           /* 0 = RGGB (the only layout supported)                     */
    int white_level;   /* e.g. 4095 for 12-bit data; 1..7281.  Every sample must   */
                       /* lie in [0, white_level]: the exact integer sums of the   */
                       /* alignment are sized for it (larger samples give        */
                       /* unspecified vectors)                                    */
    int black_level;   /* must be 0 (the synthetic data has none)                  */
} hmfsr_burst_desc;

/* Tile alignment (Sec. 3.2: coarse-to-fine pyramid block matching, then Lucas-Kanade). */
typedef struct {
    int tile;          /* raw px: 8, 16, 32 or 64; tiles are tile/2 px at every level */
    int n_levels;      /* maximum pyramid levels, 1..4 (factors 2, 4, 4 between   */
                       /* levels; a level is added while both sides stay >= 16 px) */
    int radius[4];     /* search radius per level (index 0 = finest), 0..7         */
    int lk_iters;      /* Lucas-Kanade iterations (the paper uses 3), 0..16        */
} hmfsr_align_params;

/* Merge tuning (Sec. 5; supplement S.1 heuristics and S.2 values). */
typedef struct {
    float k_detail, k_denoise, d_th, d_tr, k_stretch, k_shrink; /* kernel shape (S.1)    */
    float t, s1, s2, m_th;          /* robustness threshold, scales, motion threshold   */
    float noise_a, noise_b;         /* noise variance = noise_a * x + noise_b (DN^2)    */
    int tile;                       /* raw px of the motion field's tiles: 8, 16, 32, 64 */
} hmfsr_merge_params;

enum {
    HMFSR_OP_ALIGN = 0,
    HMFSR_OP_MERGE = 1,
    HMFSR_OP_MERGE_STAGES = 2,
    HMFSR_OP_MERGE_BACKWARD = 3,
    HMFSR_OP_ALIGN_MERGE = 4
};

/* Bytes of scratch the op needs for this burst (0 on invalid arguments).  For
 * HMFSR_OP_ALIGN, `tile` is the alignment tile; scale_num/scale_den are ignored.  For the
 * merge ops, `tile` is the motion field's tile.  The workspace must be 256-byte aligned. */
size_t hmfsr_workspace_size(int op, const hmfsr_burst_desc *desc, int tile, int scale_num, int scale_den);

/* align(burst, ref) -> motion field (Sec. 3.2).
 *   motion_dev      float32 [n_frames][TY][TX][2], written (raw px; base frame = 0).
 *   motion_int_dev  optional int32 [n_frames][TY][TX][2]: the integer block-matching
 *                   vectors in half-res px (before Lucas-Kanade); NULL to skip. */
hmfsr_status hmfsr_align(const uint16_t *burst_dev, const hmfsr_burst_desc *desc,
                         const hmfsr_align_params *params, float *motion_dev, int32_t *motion_int_dev,
                         void *ws, size_t ws_bytes, void *stream);

/* hmfsr_align with the subpixel step the paper explored before Lucas-Kanade (Sec. 3.2): a
 * quadratic fit to the block-matching error.  After the same pyramid search, each tile's
 * exact level-0 SSD at its integer vector u and at the two neighbours along each axis give
 * per axis the vertex of the parabola through the three, (E- - E+) / (2 (E- - 2 E0 + E+)),
 * 0 unless that curvature is positive, clamped to [-1/2, 1/2]; motion = 2 (u + vertex)
 * raw px, computed in FP64.  params->lk_iters is ignored; everything else as hmfsr_align,
 * with the same workspace (HMFSR_OP_ALIGN). */
hmfsr_status hmfsr_align_quadfit(const uint16_t *burst_dev, const hmfsr_burst_desc *desc,
                                 const hmfsr_align_params *params, float *motion_dev, int32_t *motion_int_dev,
                                 void *ws, size_t ws_bytes, void *stream);

/* merge(burst, motion, params, scale) -> RGB (Sec. 5, Eq. 1-9 and supplement S.1): per
 * frame, kernel covariances from the half-res structure tensor (Eq. 3-4), robustness from
 * local statistics, the noise model and the motion prior (Eq. 5-9), then per-channel
 * kernel regression of every Bayer sample over the 3x3 neighbourhood (Eq. 1-2) and a
 * final normalisation.  scale_num/scale_den in {1/1, 3/2, 2/1} (any 1 <= num/den <= 4
 * with num, den <= 8 is accepted).
 *   rgb_dev  float32 [3][Ho][Wo], written.
 *   den_dev  optional float32 [3][Ho][Wo]: per channel, log2 of the accumulated weight
 *            sum(w * Rhat) of Eq. 1's denominator (NULL to skip). */
hmfsr_status hmfsr_merge(const uint16_t *burst_dev, const hmfsr_burst_desc *desc, const float *motion_dev,
                         const hmfsr_merge_params *params, int scale_num, int scale_den, float *rgb_dev,
                         float *den_dev, void *ws, size_t ws_bytes, void *stream);

/* align + merge of one burst in one call (Sec. 3.2, then Sec. 5): the same outputs, bit
 * for bit, as hmfsr_align followed by hmfsr_merge with these arguments.  The part of the
 * merge that needs no motion (the 3x3 guide sums, the base frame's local statistics and
 * the kernel covariances of Eq. 3-4) runs on `stream` while the alignment runs beside it
 * on a library-owned stream of the highest priority (one per device and calling host
 * thread, created on first use and kept until the thread exits); events join the two
 * before the robustness (Eq. 5-9) and the accumulation (Eq. 1-2).  The call is ordered
 * on `stream` like every other entry point and may be captured into a CUDA graph once
 * the thread has made one call outside capture (the first call creates the side stream
 * and its two events).  Two calls from one host thread share that stream, so their
 * alignments run in call order.  `stream` must belong to the current device.
 *   aparams->tile must equal mparams->tile (HMFSR_ERR_INVALID_ARG otherwise).
 *   motion_dev      float32 [n_frames][TY][TX][2], written, as hmfsr_align's.
 *   motion_int_dev  optional, as hmfsr_align's.
 *   rgb_dev, den_dev as hmfsr_merge's.
 *   Workspace: hmfsr_workspace_size(HMFSR_OP_ALIGN_MERGE, desc, tile, num, den) bytes,
 *   256-byte aligned: the alignment's and the merge's scratch side by side. */
hmfsr_status hmfsr_align_merge(const uint16_t *burst_dev, const hmfsr_burst_desc *desc,
                               const hmfsr_align_params *aparams, const hmfsr_merge_params *mparams, int scale_num,
                               int scale_den, float *motion_dev, int32_t *motion_int_dev, float *rgb_dev,
                               float *den_dev, void *ws, size_t ws_bytes, void *stream);

/* hmfsr_merge in two halves that share the workspace (same ws, desc and params):
 * prepare writes the per-frame planes (kernel covariances, robustness) into ws;
 * accumulate then runs the kernel regression and normalisation from those planes.
 * hmfsr_merge == prepare + accumulate.  Useful to time or overlap the halves. */
hmfsr_status hmfsr_merge_prepare(const uint16_t *burst_dev, const hmfsr_burst_desc *desc, const float *motion_dev,
                                 const hmfsr_merge_params *params, void *ws, size_t ws_bytes, void *stream);
hmfsr_status hmfsr_merge_accumulate(const uint16_t *burst_dev, const hmfsr_burst_desc *desc, const float *motion_dev,
                                    const hmfsr_merge_params *params, int scale_num, int scale_den, float *rgb_dev,
                                    float *den_dev, void *ws, size_t ws_bytes, void *stream);

/* Bounded-memory merge (Sec. 6 and Table 2: memory that does not grow with the frame
 * count): the same outputs, bit for bit, as hmfsr_merge with these arguments, computed
 * chunk_frames non-base frames at a time.  Each chunk's frames and the base frame are
 * copied into a packed sub-burst in the workspace, their planes (kernel covariances,
 * robustness) are prepared there, and the accumulation continues from the running sums
 * of the earlier chunks: per output pixel and channel the numerator, the denominator
 * and the exponent shift, 9 floats, kept in the workspace between chunks.  The frames
 * are merged in hmfsr_merge's order (the base frame, then the others in order), so the
 * sums are the same.  The closed-form noise model only (no hmfsr_merge_options).
 *   chunk_frames  1..4096: non-base frames per chunk.
 *   Workspace: hmfsr_merge_chunked_workspace_size(desc, tile, num, den, chunk_frames)
 *   bytes, 256-byte aligned; for n_frames > chunk_frames it does not depend on n_frames.
 *   Other arguments and errors as hmfsr_merge. */
size_t hmfsr_merge_chunked_workspace_size(const hmfsr_burst_desc *desc, int tile, int scale_num, int scale_den,
                                          int chunk_frames);
hmfsr_status hmfsr_merge_chunked(const uint16_t *burst_dev, const hmfsr_burst_desc *desc, const float *motion_dev,
                                 const hmfsr_merge_params *params, int scale_num, int scale_den, int chunk_frames,
                                 float *rgb_dev, float *den_dev, void *ws, size_t ws_bytes, void *stream);

/* The per-frame merge stages alone, for inspection and testing (Sec. 5.1.2 and 5.2):
 *   omega_dev  optional float32 [n_frames][3][height/2][width/2]: the kernel covariance
 *              entries (Oxx, Oxy, Oyy) in raw px^2 at each half-res pixel (Eq. 4).
 *   rhat_dev   optional float32 [n_frames][height/2][width/2]: the final robustness Rhat
 *              (Eq. 9) of each frame on the base frame's half-res grid (1 for the base). */
hmfsr_status hmfsr_merge_stages(const uint16_t *burst_dev, const hmfsr_burst_desc *desc, const float *motion_dev,
                                const hmfsr_merge_params *params, float *omega_dev, float *rhat_dev,
                                void *ws, size_t ws_bytes, void *stream);

/* Adjoint of hmfsr_merge (reverse mode of Eq. 1-9 and the supplement's heuristics S.1)
 * for fitting the tuning parameters and the motion by gradient descent.  Given the
 * forward's outputs rgb_dev and den_dev (hmfsr_merge with den_dev, same arguments) and
 * grad_rgb_dev = dL/drgb (float32 [3][Ho][Wo]), writes
 *   grad_params_dev  float32 [8]: dL/d{k_detail, k_denoise, d_th, d_tr, k_stretch,
 *                    k_shrink, s2, t} (s2 is the robustness scale of Eq. 8 where the
 *                    motion prior does not fire; s1 is not differentiated);
 *   grad_motion_dev  float32 [n_frames][TY][TX][2]: dL/dmotion (0 for the base frame).
 * Discrete decisions (window centres, tiles, s1/s2 selection, clamps, the 5x5 argmin)
 * carry no gradient.  The forward is recomputed from the burst; the reduction order is
 * fixed, so results are deterministic.  Workspace: HMFSR_OP_MERGE_BACKWARD.  Like
 * hmfsr_align_merge, the call runs independent parts on the calling thread's side stream
 * (the kernel-shape derivatives beside the preparation, the robustness derivatives beside
 * the main adjoint kernel), joined by events: it is ordered on `stream`, and may be
 * captured once the thread has made one call of either outside capture. */
hmfsr_status hmfsr_merge_backward(const uint16_t *burst_dev, const hmfsr_burst_desc *desc, const float *motion_dev,
                                  const hmfsr_merge_params *params, int scale_num, int scale_den,
                                  const float *rgb_dev, const float *den_dev, const float *grad_rgb_dev,
                                  float *grad_params_dev, float *grad_motion_dev, void *ws, size_t ws_bytes,
                                  void *stream);

/* hmfsr_merge_backward that reuses the forward's per-frame planes: `ws` (sized for
 * HMFSR_OP_MERGE_BACKWARD) was the workspace of an hmfsr_merge call with the same burst,
 * desc, motion, params and scale, and nothing has written it since.  hmfsr_merge lays
 * its planes at the start of the workspace, where the adjoint looks for them, so the
 * preparation (kernel covariances, robustness) is not recomputed; results are those of
 * hmfsr_merge_backward.  The library cannot check the precondition. */
hmfsr_status hmfsr_merge_backward_prepared(const uint16_t *burst_dev, const hmfsr_burst_desc *desc,
                                           const float *motion_dev, const hmfsr_merge_params *params, int scale_num,
                                           int scale_den, const float *rgb_dev, const float *den_dev,
                                           const float *grad_rgb_dev, float *grad_params_dev, float *grad_motion_dev,
                                           void *ws, size_t ws_bytes, void *stream);

/* hmfsr_merge without a workspace argument, for callers that cannot allocate device
 * memory where they merge (inside another framework's memory pool, on a real-time
 * capture path where cudaMalloc could stall other streams, or behind a plugin interface
 * that passes only input and output buffers).  The paper has no counterpart; this is a
 * deployment convenience.  The call allocates nothing: its scratch is one fixed 32 MiB
 * array inside the library (held by every GPU that loads the library, until the process
 * exits).  Bursts whose merge needs more scratch than that, as hmfsr_workspace_size
 * (HMFSR_OP_MERGE, ...) reports, are rejected with HMFSR_ERR_WORKSPACE before any launch
 * (8 frames of 768 x 512 fit).  The first call on a device looks up the array's device
 * address; make that first call before capturing a stream into a CUDA graph.  The
 * address is kept for the life of the process, so after cudaDeviceReset on a device (a
 * reset ends the context the address belongs to) this entry point must not be called
 * on that device again.  All calls
 * share the one array: calls that overlap on the GPU (other streams, other host threads)
 * race and must be serialised by the caller.  Arguments and results are otherwise those
 * of hmfsr_merge. */
hmfsr_status hmfsr_merge_static(const uint16_t *burst_dev, const hmfsr_burst_desc *desc, const float *motion_dev,
                                const hmfsr_merge_params *params, int scale_num, int scale_den, float *rgb_dev,
                                float *den_dev, void *stream);

/* ---------------------------------------------------------------------------------
 * Ragged batches: many bursts (any sizes, frame counts and output scales) aligned and
 * merged by ONE persistent kernel launch, captured in a CUDA graph and replayed.
 * Results are bit-identical to hmfsr_align + hmfsr_merge on each burst.
 * Batched bursts use tile 16 and search radii 1..4 at every level.
 * --------------------------------------------------------------------------------- */
typedef struct hmfsr_batch_plan_t *hmfsr_batch_plan;

/* Plan a batch (host work only; the plan is host memory owned by the library, released
 * by hmfsr_batch_free).  Per burst b: descs[b], mparams[b], aparams[b] and the output
 * scale scale_num[b] / scale_den[b]. */
hmfsr_status hmfsr_batch_plan_create(const hmfsr_burst_desc *descs, int n_bursts, const hmfsr_merge_params *mparams,
                                     const hmfsr_align_params *aparams, const int *scale_num, const int *scale_den,
                                     hmfsr_batch_plan *out);

/* Bytes of workspace (256-byte aligned) a run of this plan needs. */
size_t hmfsr_batch_workspace_size(hmfsr_batch_plan plan);

/* Run the batch on `stream`: bursts_dev[b] (uint16, layout of desc b), rgb_dev[b]
 * (float32 [3][Ho][Wo], written) and optionally motion_dev[b] (float32 [n][TY][TX][2],
 * written; NULL array or entries: kept in the workspace).  Host arrays of device
 * pointers.  The first run, or a run with a different workspace, stream or grid,
 * captures and instantiates the CUDA graph; later runs replay it.  The call returns
 * after enqueueing; hmfsr_batch_wait reports the outcome. */
hmfsr_status hmfsr_batch_run(hmfsr_batch_plan plan, const uint16_t *const *bursts_dev, float *const *motion_dev,
                             float *const *rgb_dev, void *ws, size_t ws_bytes, void *stream);

/* Wait for the stream and return the batch's device status: HMFSR_OK, or
 * HMFSR_ERR_TIMEOUT if a block's bounded wait for a dependency ran out (the kernel then
 * stops early and the outputs are incomplete; the device stays usable). */
hmfsr_status hmfsr_batch_wait(hmfsr_batch_plan plan, void *ws, void *stream);

/* Per-stage profile of the persistent kernel (a diagnostic; off by default).  With
 * `enable` != 0 the next runs' persistent kernel has each block's lead thread add, per
 * stage, the SM clock cycles it spent waiting for the stages an item depends on and the
 * cycles the item ran, and count the items (the graph is captured again when the
 * setting changes; the graph mode records nothing).  hmfsr_batch_stage_profile copies
 * the last run's counters from workspace `ws` to the host array out[n_out], n_out >= 3 x
 * 14: for stage s = 0..13 (luminance, preparation, pyramid levels 1-3, block matching on
 * levels 3-0, Lucas-Kanade, motion prior, robustness, accumulation, unused) out[3 s] wait
 * cycles, out[3 s + 1] run cycles, out[3 s + 2] items; it synchronises `stream`. */
hmfsr_status hmfsr_batch_set_profile(hmfsr_batch_plan plan, int enable);
hmfsr_status hmfsr_batch_stage_profile(hmfsr_batch_plan plan, const void *ws, unsigned long long *out, int n_out,
                                       void *stream);

/* The integer block-matching vectors (Sec. 3.2, level 0, in half-res px) that the last
 * run of the plan on workspace `ws` computed for burst `burst`: int32
 * [n_frames][TY][TX][2] into motion_int_dev (4-byte aligned, caller-owned), as
 * hmfsr_align's motion_int_dev.  An asynchronous device-to-device copy on `stream`,
 * ordered after the run when given the run's stream.  HMFSR_ERR_INVALID_ARG for a NULL
 * plan, workspace or destination, or a burst index outside the plan. */
hmfsr_status hmfsr_batch_vectors(hmfsr_batch_plan plan, const void *ws, int burst, int32_t *motion_int_dev,
                                 void *stream);

/* Settings: accumulation work item of merge_tile_w x (128 / merge_tile_w) output pixels
 * (merge_tile_w divides 128), ctas_per_sm persistent blocks per SM (0 = as many as fit),
 * regs_variant (kernel build with 0: 128, 1: 80, 2: 64 registers per thread),
 * queue_order (0: stage-major, 1: burst-major, 2: wavefront), spin_limit polls per dependency wait
 * before HMFSR_ERR_TIMEOUT, and inject_stall != 0 to add a dependency nothing satisfies
 * (for testing the timeout path). */
hmfsr_status hmfsr_batch_configure(hmfsr_batch_plan plan, int merge_tile_w, int ctas_per_sm, int regs_variant,
                                   int queue_order, int spin_limit, int inject_stall);

/* Execution mode: 0 = the one persistent kernel (default); k > 0 = a CUDA graph of every
 * burst's own kernel sequence (the per-burst path) spread over k parallel branches. */
hmfsr_status hmfsr_batch_set_mode(hmfsr_batch_plan plan, int streams);

/* Autotuner: times the batch on the given buffers for 8 candidates -- the persistent
 * kernel at 128 registers per thread with accumulation tiles 32x4 and 16x8 (for scales
 * other than 1; scale 1 always takes 2 x 2 pixel blocks), at 80 and at 64 registers
 * (32x4), and at 128 registers with the wavefront queue; and the per-burst graph on 2, 4
 * and 8 branches -- keeps the fastest in the plan and returns its time (ms) in *best_ms
 * and every candidate's time in tune_log[8] (both nullable).  Overwrites the outputs. */
hmfsr_status hmfsr_batch_tune(hmfsr_batch_plan plan, const uint16_t *const *bursts_dev, float *const *motion_dev,
                              float *const *rgb_dev, void *ws, size_t ws_bytes, void *stream, float *best_ms,
                              float *tune_log);

void hmfsr_batch_free(hmfsr_batch_plan plan);

/* ---- Noise-dependent tuning (supplement: "Noise-dependent Tuning" and "Tuning
 * Procedure and Parameters").  The paper picks its kernel parameters and tile size from
 * one input, the base frame's SNR, estimated from the mean brightness and the noise
 * model (Sec. 5.2.2).  ---- */

/* Exact sum of every sample of frame `frame` (width x height, row stride pitch_elems),
 * written to *sum_dev, one 8-byte-aligned unsigned 64-bit integer in device memory that
 * the call zeroes first on `stream`.  mean = sum / (width * height).  Asynchronous;
 * HMFSR_ERR_INVALID_ARG for a bad frame index, size or pointer. */
hmfsr_status hmfsr_frame_sum(const uint16_t *burst_dev, const hmfsr_burst_desc *desc, int frame,
                             unsigned long long *sum_dev, void *stream);

/* ---- Monte-Carlo noise statistics (Sec. 5.2.2: the modelled sigma_md and d_md are
 * obtained "through a series of Monte Carlo simulations for different brightness
 * levels", so that clipping near the white point is accounted for).  ---- */
#define HMFSR_NOISE_LEVELS 129
#define HMFSR_NOISE_TRIALS 4096

/* Fills table_dev (device, 16-byte aligned, HMFSR_NOISE_LEVELS x 4 floats) for the noise
 * model var(x) = noise_a x + noise_b and white level WL.  Level i is brightness
 * x_i = i WL / (HMFSR_NOISE_LEVELS - 1); each of HMFSR_NOISE_TRIALS trials draws two
 * independent constant 3x3 patches of guide pixels (red/blue: one raw sample; green: the
 * mean of two), each raw sample clamp(floor(x + sqrt(var(x)) z + 1/2), 0, WL) with z an
 * Irwin-Hall normal (12 uniforms - 6) from Philox-4x32-10.  Entry i holds the trial means
 * {3x3 population variance of patch 1, red/blue; the same, green; squared difference of
 * the two patch means, red/blue; the same, green}: sigma_md^2 and d_md^2 of Eq. 6.
 * Asynchronous; deterministic up to the order of FP64 sums.  HMFSR_ERR_INVALID_ARG for a
 * NULL or misaligned table, a negative or non-finite coefficient, or WL outside 1..65535. */
hmfsr_status hmfsr_noise_table(float noise_a, float noise_b, int white_level, float *table_dev, void *stream);

/* hmfsr_merge with the robustness's modelled statistics (Eq. 6) taken from a table made
 * by hmfsr_noise_table (for this burst's noise model and white level), linearly
 * interpolated at the base frame's local mean, instead of the closed form.  Same
 * arguments, workspace size (HMFSR_OP_MERGE) and errors as hmfsr_merge; noise_table_dev
 * must be non-NULL and 16-byte aligned. */
hmfsr_status hmfsr_merge_noise(const uint16_t *burst_dev, const hmfsr_burst_desc *desc, const float *motion_dev,
                               const hmfsr_merge_params *params, const float *noise_table_dev, int scale_num,
                               int scale_den, float *rgb_dev, float *den_dev, void *ws, size_t ws_bytes,
                               void *stream);

/* ---- Options of the merge beyond hmfsr_merge_params.  ---- */
typedef struct {
    /* NULL: the closed-form noise statistics of Eq. 6; else a table from
     * hmfsr_noise_table (device, 16-byte aligned) for this burst's noise model and WL */
    const float *noise_table;
    /* 0: off; else kappa of the high-frequency artifact rejection (supplement, High
     * Frequency Artifacts Removal): a base texel whose 3x3 local means keep less than
     * kappa of its 3x3 local variance (R, G, B summed, exact integer sums, FP64 test) is
     * rejected (R = 0) in every frame whose tile there has a motion span M > m_th
     * (Eq. 7).  0.03 sits between a pattern at the guide's Nyquist frequency (~0.012) and
     * pure noise (~0.05). */
    float hf_loss;
} hmfsr_merge_options;

/* hmfsr_merge with the options above (all zero: exactly hmfsr_merge).  Same arguments,
 * workspace size (HMFSR_OP_MERGE) and errors; HMFSR_ERR_INVALID_ARG also for a NULL
 * `opts`, a misaligned table or a negative or non-finite hf_loss. */
hmfsr_status hmfsr_merge_ex(const uint16_t *burst_dev, const hmfsr_burst_desc *desc, const float *motion_dev,
                            const hmfsr_merge_params *params, const hmfsr_merge_options *opts, int scale_num,
                            int scale_den, float *rgb_dev, float *den_dev, void *ws, size_t ws_bytes, void *stream);

/* Host-only (no GPU): from the base frame's mean sample value, mean = sample_sum /
 * sample_count in DN (sample_sum from hmfsr_frame_sum, sample_count = height x width;
 * the quotient is taken here, correctly rounded in FP64), and the noise model var(x) =
 * noise_a * x + noise_b, SNR = mean / sqrt(noise_a * mean + noise_b) (one raw sample of
 * one frame; +infinity for a noise-free model), then every parameter of
 * *mparams and *aparams:
 *   k_detail 0.33 -> 0.25, k_denoise 5 -> 3, d_th 0.010 -> 0.001, d_tr 0.020 -> 0.006,
 *   linear in SNR from SNR <= 6 (the denoising end) to SNR >= 30 (the detail end);
 *   tile 64 for SNR < 10, 32 for SNR < 14, else 16 (both structs);
 *   k_stretch 4, k_shrink 2, t 0.12, s1 12, s2 2, m_th 0.8, noise_a/b as given;
 *   alignment: 4 levels, radii 1 (finest), 4, 4, 4, 3 Lucas-Kanade iterations.
 * `snr` may be NULL.  HMFSR_ERR_INVALID_ARG for sample_count 0, a sum or count of 2^53 or
 * more, a negative or non-finite noise coefficient, or a NULL struct. */
hmfsr_status hmfsr_snr_tuning(uint64_t sample_sum, uint64_t sample_count, float noise_a, float noise_b,
                              hmfsr_merge_params *mparams, hmfsr_align_params *aparams, double *snr);

/* ---- Measurement aid (not part of the method).  The accumulation (Eq. 1-2) is bound
 * by FP32 and MUFU issue rather than by HBM, so its roofline divides by this GPU's
 * measured FP32 fused-multiply-add rate and ex2 rate.  ---- */
enum { HMFSR_PIPE_FP32_FMA = 0, HMFSR_PIPE_MUFU_EX2 = 1 };

/* Enqueues one issue-rate probe on `stream`: `blocks` blocks of 256 threads, each thread
 * running 8 independent chains of `iters` x 16 dependent operations (pipe
 * HMFSR_PIPE_FP32_FMA: fmaf; HMFSR_PIPE_MUFU_EX2: ex2.approx.ftz).  *lane_ops (nullable)
 * receives the operations the launch performs (blocks x 256 x iters x 128); the caller
 * times the launch with events on `stream`.  sink_dev: 256 floats of device memory
 * (4-byte aligned), written only on a branch no input takes.  HMFSR_ERR_INVALID_ARG for
 * an unknown pipe, blocks outside [1, 2^20], iters outside [1, 2^24] or a NULL or
 * misaligned sink. */
hmfsr_status hmfsr_pipe_probe(int pipe, int blocks, int iters, float *sink_dev, double *lane_ops, void *stream);

/* ---- Checked build (the library compiled with -DHMFSR_CHECKED: a test build, not the
 * default).  The paper has no counterpart; this is a memory-safety aid.  In that build
 * every global load and store of the alignment and merge kernels (the entry points
 * hmfsr_align, hmfsr_align_quadfit, hmfsr_merge and its variants _ex, _noise, _prepare,
 * _accumulate, _stages and _static) is checked against the buffers of its call: the
 * burst, motion, outputs, tables and the workspace the call needs.  An access outside
 * all of them is not made (a load gives 0, a store is dropped) and the source line of
 * the first such access goes to a device error word; nothing traps.  Calls that overlap
 * on the GPU share the checker's state.  In the default build both functions return
 * HMFSR_ERR_UNSUPPORTED.  ---- */

/* *line = the error word (0: every checked access stayed inside its call's buffers);
 * with reset != 0 the word is cleared.  Synchronises with the device (legacy default
 * stream). */
hmfsr_status hmfsr_check_status(int reset, int *line);

/* Test hook: every workspace registered from now on is taken as `bytes` shorter than
 * the call needs, so that the kernels' last workspace accesses count as outside (they
 * are then not made).  0 restores the exact extent. */
hmfsr_status hmfsr_check_shrink(size_t bytes);

/* Human-readable name of a status code (static string). */
const char *hmfsr_status_string(hmfsr_status s);

/* Library version, e.g. "0.1.0" (static string). */
const char *hmfsr_version(void);

#ifdef __cplusplus
}
#endif
#endif /* HMFSR_H */
