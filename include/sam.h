/*
 * sam.h -- C ABI of the GB300 shape-based alignment detector.
 *
 * The detector follows T.-S. Le and C.-Y. Lin, "GPU-accelerated image
 * alignment for object detection in industrial applications" (arXiv
 * 2112.05576), Sec. II: edge extraction (x/y gradients and magnitudes,
 * thresholded), an image pyramid, an exhaustive (x, y, theta) search at the
 * pyramid's top level scored by the normalised gradient-direction similarity
 * of Eq. (1) over model points projected by the rigid transform of Eq. (2),
 * each point taking the best vote in its neighbouring-search window, and
 * refinement down the pyramid.
 *
 * Conventions shared by every entry point
 *   - Images are 8-bit grey, row-major, `stride` bytes between rows
 *     (stride >= width).  x grows to the right, y downwards.
 *   - "device" pointers are CUDA global-memory pointers of the current
 *     device; "host" pointers are ordinary host memory.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Every call is ordered on that stream; calls that return
 *     results to host memory synchronise it before returning.
 *   - No entry point aborts: errors are returned as sam_status, and outputs
 *     are left unspecified on error.  sam_status_str() names each code.
 *   - Thresholds are in units of |g| / 4 where g is the 3x3 Sobel gradient,
 *     so a step edge of height h has magnitude h.  A pixel is an edge iff
 *     gx^2 + gy^2 >= 16 T^2 (exact integer compare).
 *   - Angles: theta_k = k * dtheta_l, dtheta_l = angle_step_deg * 2^l at
 *     pyramid level l, k = 0 .. 360 / dtheta_l - 1 (full circle).
 *   - The template reference point is (floor(W_t/2), floor(H_t/2)) at every
 *     level; a pose (x, y, theta) puts that point at pixel (x, y).
 */
#ifndef SAM_H
#define SAM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    SAM_OK = 0,
    SAM_ERR_ARG = 1,          /* invalid argument (null pointer, bad size, bad parameter) */
    SAM_ERR_NOMEM = 2,        /* host or device allocation failed */
    SAM_ERR_CUDA = 3,         /* a CUDA runtime call or kernel launch failed */
    SAM_ERR_TIMEOUT = 4,      /* a bounded device-side wait gave up */
    SAM_ERR_EMPTY_MODEL = 5,  /* a template level has no edge point */
    SAM_ERR_CAPACITY = 6      /* a fixed-capacity device buffer would overflow */
} sam_status;

/* Field precisions of the normalised search gradients w_hat.
 * SAM_ANGLE16 (angle-only storage; the paper stores x/y gradients, this form
 * keeps their direction alone): one 16-bit code per pixel, 0x8000 | a on an
 * edge with a = round(atan2(gy, gx) * 32768 / (2 pi)) mod 32768 from the
 * integer Sobel gradient, 0 elsewhere; it stands for the unit vector
 * (cos, sin)(a 2 pi / 32768), so a term of Eq. (1) moves by at most
 * 2 sin(pi / 65536) < 9.6e-5 against the exact direction.  Code rows have
 * pitch w (SAM_LAYOUT_PIXEL) or w rounded up to a multiple of 8 codes,
 * 16-byte rows, padding codes 0 (SAM_LAYOUT_PAIRS, the layout the scorers
 * read).  Served by sam_gradient, sam_score_map and sam_score_window. */
enum { SAM_FP32 = 0, SAM_BF16 = 1, SAM_FP16 = 2, SAM_ANGLE16 = 3 };

/* Field layouts.  SAM_LAYOUT_PIXEL: each row holds w pixels, each pixel the
 * pair (wx, wy); row pitch w pixels.  SAM_LAYOUT_PAIRS: each row holds pixel
 * pairs {wx_2j, wx_2j+1, wy_2j, wy_2j+1}; row pitch w rounded up to a
 * multiple of 4 pixels, padding pixels zero.  Same bytes per pixel. */
enum { SAM_LAYOUT_PIXEL = 0, SAM_LAYOUT_PAIRS = 1 };

typedef struct sam_model sam_model;

/* Model parameters (Sec. II inputs: edge thresholds, number of pyramid
 * levels, rotation step).
 *   low, high       hysteresis thresholds for the template; `low` is also the
 *                   single threshold of the search image.  1 <= low <= high.
 *   levels          pyramid levels, 1..8; every template level must keep at
 *                   least one edge point.
 *   angle_step_deg  rotation step at level 0; 360/angle_step_deg must be an
 *                   integer divisible by 2^(levels-1).
 *   polarity        0: Eq. (1) as printed (signed cosine);
 *                   1: ignore local polarity (|cosine| per neighbour). */
typedef struct {
    int low, high;
    int levels;
    double angle_step_deg;
    int polarity;
} sam_model_params;

/* Detection parameters (Sec. II inputs: step sizes, neighbouring-search size).
 *   step_x, step_y     translation steps of the top-level exhaustive search
 *                      (>= 1; refinement below the top always uses 1 px).
 *   neighbourhood      neighbouring-search window side, 1 or 3.
 *   min_score          poses below this score are discarded at every level.
 *   max_detections     at most this many poses are returned.
 *   top_k              top-level candidates refined down the pyramid (1..1024).
 *   precision          SAM_FP32, SAM_BF16 or SAM_FP16 storage of the top-level
 *                      w_hat field; refinement and final scores are FP32.
 *   early_termination  1: stop scoring a top-level pose once the partial sum
 *                      proves M < min_score (exact-safe bound, every
 *                      remaining term is at most 1); such poses are written
 *                      as -inf in score maps. */
typedef struct {
    int step_x, step_y;
    int neighbourhood;
    float min_score;
    int max_detections;
    int top_k;
    int precision;
    int early_termination;
} sam_detect_params;

/* One detection at level 0: reference point (x, y) in pixels, rotation in
 * degrees, score M of Eq. (1) (FP32).  angle_index is k at level 0;
 * scale_index is j of a scaled model's grid (scale sam_model_scale(m, j)),
 * 0 for a rigid model. */
typedef struct {
    float x, y, theta_deg, score;
    int angle_index;
    int level0_x, level0_y;
    int scale_index;
} sam_pose;

const char *sam_status_str(sam_status s);

/* Library version and the CUDA architecture it was compiled for (e.g. 1030).
 * Library metadata; the paper has no counterpart.  Never fail. */
int sam_version(void);
int sam_compiled_arch(void);

/* Fill `p` (host, caller-owned; NULL is ignored) with defaults: low 30,
 * high 60, levels 3, angle_step 1.0, polarity 0.  The paper prints no
 * thresholds or steps for these (Sec. III names its search steps only for
 * its own samples); the values are this library's. */
void sam_default_model_params(sam_model_params *p);
/* Fill `p` (host, caller-owned; NULL is ignored) with defaults: steps 1,
 * neighbourhood 3 (the neighbouring-search size of Sec. II), min_score 0.7,
 * max_detections 16, top_k 64, FP32, early termination on. */
void sam_default_detect_params(sam_detect_params *p);

/* ---------------------------------------------------------------------------
 * Model (Sec. II: the model image's edge points at every pyramid level, and
 * per level l and angle index k the Eq. (2) projection of every point:
 * integer offset round(R(theta_k) t) and unit direction R(theta_k) g/|g|).
 * Built on the host in FP64; device tables are uploaded on first use.
 *   tmpl     host pointer, w x h bytes with row pitch `stride`.
 *   out      receives the new model; free it with sam_free_model.
 * Errors: SAM_ERR_ARG (bad sizes or params), SAM_ERR_EMPTY_MODEL,
 *         SAM_ERR_NOMEM.
 * ------------------------------------------------------------------------- */
sam_status sam_create_model(const uint8_t *tmpl, int w, int h, int stride, const sam_model_params *params,
                            sam_model **out);
void sam_free_model(sam_model *m);

/* A scaled model (Sec. II, after Eq. (2): the paper notes that other types
 * of projection could be implemented; here Eq. (2) with R(theta) replaced by
 * A = s R(theta)).  As sam_create_model, plus a grid of scales
 * s_j = scale_min + j * scale_step, j < n_scales (1 <= n_scales <= 64,
 * 0 < s_j <= 16), the same at every pyramid level.  Per level and table
 * K = j * num_angles + k the projection of each point is the integer offset
 * floor(A t + 1/2) (A = [[s c, -(s sn)], [s sn, s c]] evaluated in FP64 as
 * written) and the unit direction R(theta) g/|g|.  Score maps of a scaled
 * model have num_scales x num_angles planes (plane K); detection searches
 * the scales too (candidates are strict local maxima over the up to 80
 * neighbours in (scale, angle circular, y, x), the scale axis not circular;
 * the descent searches scale j +- 1 inside the grid with x, y and angle, up
 * to 81 poses per level; the child shift turns and scales the reference
 * offset by the parent's A) and returns each pose's scale_index.  Scaled
 * models are not served by the batched plan (sam_multi_create), the
 * continuous-pose score and refinement or the sub-pixel fit (SAM_ERR_ARG).
 * n_scales = 1 with scale_min = 1 gives the rigid model.
 * Errors: SAM_ERR_ARG, SAM_ERR_EMPTY_MODEL, SAM_ERR_NOMEM. */
sam_status sam_create_model_scaled(const uint8_t *tmpl, int w, int h, int stride, const sam_model_params *params,
                                   double scale_min, double scale_step, int n_scales, sam_model **out);
/* The scale grid (host only; the paper has no counterpart): number of
 * scales (1 for a rigid model, 0 for NULL) and s_j (0.0 for j out of range). */
int sam_model_num_scales(const sam_model *m);
double sam_model_scale(const sam_model *m, int j);

/* Model inspection (host only, no device work; the paper has no
 * counterpart).  The int getters return 0 for a NULL model or a level out of
 * range; sam_model_template_size returns 1 and writes the level's template
 * size (w, h; either pointer may be NULL) or returns 0.  num_angles counts
 * the angles of one scale; the table index k of the calls below runs over
 * num_scales x num_angles tables (k = scale j * num_angles + angle). */
int sam_model_levels(const sam_model *m);
int sam_model_num_points(const sam_model *m, int level);
int sam_model_num_angles(const sam_model *m, int level);
int sam_model_template_size(const sam_model *m, int level, int *w, int *h);
/* Copy the Eq. (2) table of (level, k) to host arrays of num_points entries:
 * integer offsets ox, oy and FP32 unit directions px, py. */
sam_status sam_model_rotated_points(const sam_model *m, int level, int k, int32_t *ox, int32_t *oy, float *px,
                                    float *py);
/* Copy the model's level points (template coordinates t relative to the
 * reference point and integer Sobel gradient), in the model's point order. */
sam_status sam_model_points(const sam_model *m, int level, int32_t *tx, int32_t *ty, int32_t *gx, int32_t *gy);
/* Coarse-to-fine child shift for a parent at level+1 with angle index k:
 * the level-`level` search centre is 2 (x, y) + (sx, sy). */
sam_status sam_model_child_shift(const sam_model *m, int level, int k_parent, int32_t *sx, int32_t *sy);

/* ---------------------------------------------------------------------------
 * Full detection (Sec. II): pyramid, gradients, top-level exhaustive search,
 * candidates, refinement to level 0, non-maximum suppression.
 *   img            w x h image, row pitch `stride`; a device pointer if
 *                  img_on_device != 0, else a host pointer.
 *   out            host array of `capacity` poses, best first.
 *   n_out          host int, receives the number of poses written.
 * With a scaled model (sam_create_model_scaled) the search also runs over
 * its scales and each pose carries its scale_index.
 * The model keeps an internal device workspace that grows to the largest
 * image seen: calls on one model must not overlap (serialise them on one
 * stream or host thread).  Synchronises `stream` before returning.
 * Errors: SAM_ERR_ARG, SAM_ERR_NOMEM, SAM_ERR_CUDA.
 * ------------------------------------------------------------------------- */
sam_status sam_detect(sam_model *m, const uint8_t *img, int w, int h, int stride, int img_on_device,
                      const sam_detect_params *params, void *stream, sam_pose *out, int capacity, int *n_out);

/* Detection (Sec. II, as sam_detect) of `count` images of equal size
 * stored back to back (image i at img + i * image_bytes, rows `stride`
 * bytes apart), all steps batched into one launch per stage.  img is a
 * device pointer if img_on_device != 0, else a host pointer: the images are
 * then copied into the model's workspace on `stream` inside the call (one
 * copy when image_bytes == stride * h; page-locked host memory makes it
 * asynchronous).  Poses of image i go to out[i * capacity ...], their count
 * to n_out[i] (host arrays, count * capacity and count entries).
 * Synchronises `stream`.  Errors as sam_detect. */
sam_status sam_detect_batch(sam_model *m, const uint8_t *img, int count, size_t image_bytes, int w, int h,
                            int stride, int img_on_device, const sam_detect_params *params, void *stream,
                            sam_pose *out, int capacity, int *n_out);

/* ---------------------------------------------------------------------------
 * Batched detection of uneven workloads (Sec. II detection applied to many
 * (image, model) pairs; the batching itself has no counterpart in the
 * paper).  A plan is built once for a batch shape -- image sizes, models and
 * pairs -- and owns every device buffer.  Each run is a fixed sequence of
 * launches over all images and pairs: pyramid steps and gradients as job
 * lists, one persistent exhaustive scorer that takes (pair, super-tile,
 * angle group) units from an atomic counter, FP32 rescoring for 16-bit
 * fields, candidates, refinement and NMS; the plan captures the sequence once
 * into a CUDA graph and replays it.
 *   models       the plan keeps the pointers; the models must outlive it and
 *                share one edge threshold and polarity.
 *   image_sizes  2 * n_images ints (w, h).
 *   pairs        n_pairs (image, model) index pairs; a model with L levels
 *                needs images of at least 2^(L-1) pixels a side.
 *   params       as for sam_detect, with step_x = step_y = 1.
 * Images are written by the caller into the plan's device buffers
 * (sam_multi_image: device pointer and row pitch of image i) before a run.
 * sam_multi_run replays the graph on `stream`, then copies every pair's poses
 * to out[i * capacity ...] and their count to n_out[i] (host, caller order)
 * and synchronises the stream.  Plans are not thread-safe; runs of one plan
 * must not overlap.  sam_multi_autotune times the scorer of the current batch
 * (images already written) over its tiling candidates (super-tile 1..2 x
 * 1..2, angles per unit 1, 3, 5, 9, 15, 4 or 8 warps, 6 or 10 pose columns
 * per thread) and keeps the fastest, writing cfg_out[5 i ..] = (sx, sy, tg,
 * warps, cols) and ms_out[i]; sam_multi_set_tiling sets one.  sam_multi_stats: top-level pose-points per
 * run (nominal), kernels per graph replay, device bytes held.
 * Errors: SAM_ERR_ARG, SAM_ERR_NOMEM, SAM_ERR_CUDA, SAM_ERR_TIMEOUT.
 * ------------------------------------------------------------------------- */
typedef struct sam_multi sam_multi;
typedef struct {
    int image, model;
} sam_pair;
sam_status sam_multi_create(sam_model *const *models, int n_models, const int32_t *image_sizes, int n_images,
                            const sam_pair *pairs, int n_pairs, const sam_detect_params *params, sam_multi **out);
void sam_multi_free(sam_multi *mp);
uint8_t *sam_multi_image(sam_multi *mp, int i, int *pitch);
/* Copy image i (w x h as declared, row pitch `stride`; device pointer if
 * on_device, else host) into the plan, ordered on `stream`. */
sam_status sam_multi_set_image(sam_multi *mp, int i, const uint8_t *src, int stride, int on_device, void *stream);
sam_status sam_multi_run(sam_multi *mp, void *stream, sam_pose *out, int capacity, int *n_out);
sam_status sam_multi_set_tiling(sam_multi *mp, int sx, int sy, int tg, int warps, int cols);
sam_status sam_multi_autotune(sam_multi *mp, void *stream, int32_t *cfg_out, float *ms_out, int max_out,
                              int *n_out);
sam_status sam_multi_stats(const sam_multi *mp, long long *pose_points, long long *graph_kernels,
                           size_t *device_bytes);
/* Copy of pair `pair`'s top-level score map, for inspection (the paper has
 * no counterpart).  The map is FP32 [nth][gh][gw], pose (x, y, theta_k) at
 * [k][y][x], and holds what the plan's last run (sam_multi_run or an
 * autotuning run) left in it: Eq. (1) scores (with a 16-bit field, the
 * scorer's 16-bit-field scores, within the storage bound 8e-4 (FP16) or 6e-3
 * (BF16) of the FP32 ones; candidate extraction decides on FP32 rescores of
 * its own), -inf for poses pruned by early termination.
 *   dst       device float array of `capacity` >= nth * gh * gw entries, or
 *             NULL to read the shape only.
 *   nth, gh, gw, level  optional host outputs: the map's shape and the
 *             pyramid level it scores.
 * The copy is ordered on `stream` (no synchronisation).  Errors: SAM_ERR_ARG
 * (NULL plan, pair out of range, capacity too small), SAM_ERR_CUDA. */
sam_status sam_multi_pair_map(const sam_multi *mp, int pair, float *dst, size_t capacity, int *nth, int *gh,
                              int *gw, int *level, void *stream);

/* ---------------------------------------------------------------------------
 * Individual steps on caller-owned device buffers (stream-ordered, no
 * synchronisation, no allocation).
 * ------------------------------------------------------------------------- */

/* Pyramid step (Sec. II, image pyramid): dst(x, y) =
 * (src(2x,2y) + src(2x+1,2y) + src(2x,2y+1) + src(2x+1,2y+1) + 2) >> 2 for
 * x < w/2, y < h/2.  src, dst device; dst pitch dst_stride >= w/2. */
sam_status sam_pyramid_down(const uint8_t *src, int w, int h, int src_stride, uint8_t *dst, int dst_stride,
                            void *stream);

/* The whole image pyramid (Sec. II) in one launch: levels 1 .. levels-1 of
 * a w x h device image, level l the pyramid step of level l - 1 (sizes
 * floor(w / 2^l) x floor(h / 2^l)), written to dst[l - 1] with row pitch
 * dst_stride[l - 1] (>= the level's width); dst and dst_stride are host
 * arrays of levels - 1 entries, the buffers device memory.  Identical to
 * levels - 1 calls of sam_pyramid_down; the detection pipeline uses it.
 * 2 <= levels <= 8.  Errors: SAM_ERR_ARG, SAM_ERR_CUDA. */
sam_status sam_pyramid_levels(const uint8_t *src, int w, int h, int src_stride, int levels, uint8_t *const *dst,
                              const int *dst_stride, void *stream);

/* Edge extraction (Sec. II) of a device image: 3x3 Sobel gx, gy (zero on the
 * 1-pixel border), edge iff gx^2+gy^2 >= 16 low^2, and the unit field
 * w_hat = g/|g| on edges, (0,0) elsewhere.
 *   field   device, h rows in `layout` (SAM_LAYOUT_PIXEL or SAM_LAYOUT_PAIRS),
 *           float components (8 B/px) for SAM_FP32, bf16 or fp16 (4 B/px)
 *           for SAM_BF16 / SAM_FP16, 16-bit angle codes (2 B/px; rows as
 *           described at SAM_ANGLE16) for SAM_ANGLE16; 16-byte aligned for
 *           SAM_LAYOUT_PAIRS.  The angle codes are computed from the integer
 *           gradient with an FP32 atan2, redone in FP64 where the FP32 value
 *           lies within 0.02 of a rounding boundary, so they equal the
 *           rounding of the exact angle.
 *   gx, gy  optional device int16 outputs (w*h, dense), NULL to skip; not
 *           with SAM_LAYOUT_PAIRS or SAM_ANGLE16. */
sam_status sam_gradient(const uint8_t *img, int w, int h, int stride, int low, int precision, int layout,
                        void *field, int16_t *gx, int16_t *gy, void *stream);

/* Exhaustive score map of one model level (Eq. (1) with the neighbouring
 * search, Eq. (2) projection, Sec. II three nested loops):
 *   map[(k * gh + gyi) * gw + gxi] = M(gxi * step_x, gyi * step_y, theta_k)
 * for k < num_angles(level), gh = ceil(h/step_y), gw = ceil(w/step_x); for
 * a scaled model k runs over the num_scales x num_angles tables (plane
 * j * num_angles + k: scale j, angle k).
 *   field   device w_hat field of the search image at that level (layout and
 *           precision as produced by sam_gradient).
 *   map     device float array of num_angles * gh * gw.
 * With early_termination, poses proved below min_score are written -inf.
 * The tiled kernel serves SAM_LAYOUT_PAIRS fields at step 1 when its
 * shared-memory window fits; everything else uses the generic kernel.
 * SAM_ANGLE16 code fields (SAM_LAYOUT_PAIRS, step 1, a template whose window
 * fits) are scored by the tiled kernel only: each CTA stages its window of
 * codes by TMA and expands it to FP32 unit vectors in shared memory (sincospi
 * in FP32, within 2.4e-7 of the FP64 decoding) before scoring; other calls
 * with codes return SAM_ERR_ARG.  With
 * early termination the tiled kernel runs in its persistent form (work units
 * of the edge-presence bound, then the surviving poses, pulled by resident
 * CTAs) with a queue taken from the device's default stream-ordered memory
 * pool (cudaMallocAsync / cudaFreeAsync on `stream`).
 * Errors: SAM_ERR_ARG, SAM_ERR_CUDA, SAM_ERR_TIMEOUT (a bounded wait for the
 * window's TMA copy gave up; checked on the next synchronising call). */
sam_status sam_score_map(sam_model *m, int level, const void *field, int w, int h, int precision, int layout,
                         int step_x, int step_y, int neighbourhood, float min_score, int early_termination,
                         float *map, void *stream);

/* A window of Eq. (1) scores at one level: the poses x0 <= x < x0 + gw,
 * y0 <= y < y0 + gh (step 1, neighbourhood 1 or 3) and angle indices
 * k0 <= k < k0 + nk, written to map[(k - k0) * gh * gw + (y - y0) * gw +
 * (x - x0)] (device, float, 8-byte aligned).  The paper has no counterpart;
 * it serves exhaustive searches too large for one score map (a full-
 * resolution search of a large template over a large image is scored slice
 * by slice) and the single-image path of the tiled scorers: `field` is the
 * level's SAM_LAYOUT_PAIRS field in `precision` (16-byte aligned, pitch
 * field_pitch(w); SAM_ANGLE16 codes: pitch w rounded up to 8 codes).
 * Templates whose rotated extent exceeds one shared-memory window are scored
 * by the chunked kernel (points grouped by 16 x 16 offset cell, one staged
 * window per cell; not for SAM_ANGLE16, which then returns SAM_ERR_ARG).
 * field32 rescoring applies to SAM_BF16 / SAM_FP16 only.  early_termination as in
 * sam_score_map (-inf for pruned poses).  For a 16-bit `precision` with a
 * non-NULL field32 (the level's FP32 SAM_LAYOUT_PIXEL field, pitch w), every
 * pose within the storage error bound of min_score is rescored in FP32 and
 * every other pose written -inf, as in sam_detect; scratch (device, 8-byte
 * aligned) of sam_score_window_scratch_bytes(R) bytes holds up to R such
 * poses, and poses beyond R are written NaN.  With early_termination the
 * chunked kernel first applies the edge-presence bound (a pose is scored
 * only if enough of its points have an edge pixel that can vote for them in
 * their neighbouring-search window): whole-image edge bitmaps and one bit
 * per pose, in scratch taken from and returned to the device's default
 * stream-ordered pool on `stream` (cudaMallocAsync / cudaFreeAsync); when
 * the pool has no room or `stream` is being captured, the bound is skipped
 * and every pose scored.  Otherwise no allocation; stream-ordered, no
 * synchronisation.  Errors: SAM_ERR_ARG (ranges, alignment,
 * nk * gw * gh >= 2^32, nk > 65535, a template no scorer's window fits),
 * SAM_ERR_CUDA. */
size_t sam_score_window_scratch_bytes(size_t max_rescored);
sam_status sam_score_window(sam_model *m, int level, const void *field, int w, int h, int precision, int x0, int y0,
                            int gw, int gh, int k0, int nk, int neighbourhood, float min_score, int early_termination,
                            const float *field32, void *scratch, size_t scratch_bytes, float *map, void *stream);

/* Score-kernel selection and tiling, process-wide (autotuner hook; the paper
 * has no counterpart).  kernel: 0 automatic, 1 generic one-thread-per-pose,
 * 2 tiled (falls back to generic when the tiled kernel cannot serve a call).
 * A thread scores an 8 x cols block of poses of one angle (cols 6 or 10);
 * a warp tile is (8 x cols) x 32 poses for FP32 fields, (16 x cols) x 16 for
 * 16-bit fields.  sx, sy: CTA super-tile in warp tiles; tg: angles per CTA,
 * or 0 for the chunked tiled kernel (one angle per CTA, points grouped by
 * 16 x 16 offset cell with one staged window per cell; requires
 * sx * sy == warps and cols 6); warps: 4 or 8.  Returns SAM_ERR_ARG on
 * out-of-range values. */
sam_status sam_set_score_kernel(int kernel, int sx, int sy, int tg, int warps, int cols);
/* Reads back the current selection (any pointer may be NULL). */
void sam_get_score_kernel(int *kernel, int *sx, int *sy, int *tg, int *warps, int *cols);

/* Autotuner for the tiled exhaustive scorer (the paper has no counterpart).
 * Prepares the top-level field of the caller's batch (arguments as for
 * sam_detect_batch, images on the device), then times the tiled kernel with
 * every tiling of its candidate set (super-tile 1..3 x 1..2 warp tiles,
 * angles per CTA 1, 2, 3, 4, 5, 6, 8, 9, 11, 12, 15, 23 or all, 4 or 8
 * warps, 6 or 10 pose columns
 * per thread; tilings whose window does not fit are skipped) and the
 * chunked kernel with its CTA tiles (2x2, 4x1, 1x4 of 4 warps; 2x4, 4x2 of
 * 8 warps; reported with tg = 0) using CUDA events on `stream`, and keeps
 * the fastest for this model, this field precision and this batch class
 * (count 1, or more than 1; used by later calls with that precision and
 * class -- or the other class when only that one is tuned -- while
 * sam_set_score_kernel selects 0, automatic).
 * Optional outputs: cfg_out[5 i ..] = (sx, sy, tg, warps, cols) and
 * ms_out[i] of up to max_out candidates; *n_out = how many were written.  Uses the model's workspace; synchronises `stream`.
 * Errors: SAM_ERR_ARG, SAM_ERR_NOMEM, SAM_ERR_CUDA, SAM_ERR_TIMEOUT. */
sam_status sam_autotune(sam_model *m, const uint8_t *img, int count, size_t image_bytes, int w, int h, int stride,
                        const sam_detect_params *params, void *stream, int32_t *cfg_out, float *ms_out, int max_out,
                        int *n_out);
/* The tiling the model's next calls with field `precision` over `count`
 * images will use (a process-wide selection set by sam_set_score_kernel
 * overrides the model's tuning; tuned, else the default; the paper has no
 * counterpart).
 * All outputs host ints.  Errors: SAM_ERR_ARG (NULL model or output,
 * precision out of range, count < 1). */
sam_status sam_model_tiling(const sam_model *m, int precision, int count, int32_t *sx, int32_t *sy, int32_t *tg,
                            int32_t *warps, int32_t *cols);
/* Self-test of failure detection (the paper has no counterpart): one warp
 * waits on an mbarrier that nothing completes, with the scorers' bounded
 * wait limited to limit_us microseconds (1 .. 10^6; the scorers use 1 s),
 * and reports the give-up through the device error flag as the scorers do.
 * No copy is issued, so nothing is left in flight.  Returns SAM_ERR_TIMEOUT
 * (the expected outcome; the flag is read and cleared) with the time the
 * wait took in *waited_ms (may be NULL); SAM_OK would mean the wait
 * completed.  Synchronises the device.  Errors: SAM_ERR_ARG, SAM_ERR_NOMEM,
 * SAM_ERR_CUDA. */
sam_status sam_selftest_wait_timeout(int limit_us, double *waited_ms);
/* The same for the other bounded wait of the tiled scorer: in its persistent
 * form a CTA that has claimed a task of surviving poses waits (1 s limit)
 * until the CTA producing it publishes it.  Here one thread waits for a task
 * whose flag nothing sets, in a list whose one work unit never completes,
 * limited to limit_us; returns as sam_selftest_wait_timeout. */
sam_status sam_selftest_task_wait_timeout(int limit_us, double *waited_ms);

/* Device-side error flag of the tiled kernel's bounded waits (failure
 * detection; the paper has no counterpart): returns 1 and clears it if any
 * wait gave up since the last call, else 0 (synchronises the device). */
int sam_take_device_error(void);

/* Candidates of a scaled model's map [n_scales * n_angles][gh][gw] (plane
 * j * n_angles + k for scale j, angle k; generalises sam_candidates, the
 * paper has no scale axis): poses with score >= min_score that beat each
 * of their up to 80 neighbours in (scale j +- 1 inside the grid, angle
 * circular, y, x), the best K (1 <= K <= 1024) by the same order, written as
 * (plane, y, x) triples to out_kyx.  Scratch: device buffer of
 * sam_candidates_scaled_scratch_bytes(n_scales, n_angles, gh, gw) bytes.
 * n_scales = 1 is sam_candidates.  Stream-ordered, no synchronisation.
 * Errors: SAM_ERR_ARG, SAM_ERR_CUDA. */
size_t sam_candidates_scaled_scratch_bytes(int n_scales, int n_angles, int gh, int gw);
sam_status sam_candidates_scaled(const float *map, int n_scales, int n_angles, int gh, int gw, float min_score, int K,
                                 int32_t *out_kyx, float *out_s, int *count, void *scratch, void *stream);

/* Candidate extraction from a score map [nth][gh][gw] (Sec. II returns the
 * best pose; for several instances this library reads it as the local
 * maxima): poses with score >= min_score that beat all 26 neighbours in
 * (theta circular, y, x) under the order (higher score, then smaller
 * (k, y, x)), the best K of them (1 <= K <= 1024).  Stream-ordered, no
 * synchronisation.  Errors: SAM_ERR_ARG (NULL pointers, sizes, K),
 * SAM_ERR_CUDA.
 *   out_kyx  device int32 array of 3*K: (k, y, x) per candidate, best first.
 *   out_s    device float array of K.
 *   count    device int, receives min(K, number of local maxima).
 *   scratch  device buffer of sam_candidates_scratch_bytes(nth, gh, gw). */
size_t sam_candidates_scratch_bytes(int nth, int gh, int gw);
sam_status sam_candidates(const float *map, int nth, int gh, int gw, float min_score, int K, int32_t *out_kyx,
                          float *out_s, int *count, void *scratch, void *stream);

/* sam_candidates without a scratch argument and without any allocation (the
 * paper has no counterpart; this exists for callers that cannot call
 * cudaMalloc when they need candidates -- a deadline-bound control loop, where
 * cudaMalloc's latency and implicit device synchronisation are not allowed,
 * or an integration whose device memory is fixed at start-up).  Same inputs,
 * outputs and results as sam_candidates.  Its scratch is a 4 MiB array in
 * the library's device memory (held by every GPU that loads the library
 * until exit); maps with sam_candidates_scratch_bytes(nth, gh, gw) above
 * 4 MiB are rejected with SAM_ERR_CAPACITY.  The first call on a device looks
 * up that array's device address (with the device current) and caches it
 * with the id of the device's context; make that first call before any
 * stream capture.  After a device reset (a new primary context) the next
 * call looks the address up again, so it too must come before any capture.  All calls share the array
 * and leave their contents in it (the counter is cleared at the start of
 * each call): calls whose GPU work overlaps race and must be serialised by
 * the caller.  Errors: SAM_ERR_ARG, SAM_ERR_CAPACITY, SAM_ERR_CUDA. */
sam_status sam_candidates_noalloc(const float *map, int nth, int gh, int gw, float min_score, int K,
                                  int32_t *out_kyx, float *out_s, int *count, void *stream);

/* ---------------------------------------------------------------------------
 * Differentiable score on continuous poses (an extension: the paper scores
 * integer poses only).  For pose (x, y, theta) -- x, y in pixels of the
 * model level's image, theta in degrees -- every model point t_i of that
 * level is placed at p_i = R(theta) t_i + (x, y) (Eq. (2) without rounding),
 * its unit direction turned to d_i = R(theta) g_i/|g_i|, and the unit search
 * field is sampled at p_i by bilinear interpolation of the four surrounding
 * pixels (pixels outside the image count as (0, 0)):
 *   M_c = (1/n) sum_i d_i . w_bil(p_i)       (polarity 1: |d_i . w_bil(p_i)|)
 * (Eq. (1) at a continuous pose, without the neighbourhood maximum, which is
 * not differentiable).  Its derivatives are those of the bilinear sample
 * inside each pixel cell (one-sided at cell borders: the cell of floor(p)).
 *
 * Fields are FP32 unit fields in SAM_LAYOUT_PIXEL as written by sam_gradient
 * (interleaved (wx, wy), row pitch `pitch` pixels >= w; device memory, 8-byte
 * aligned), one per search image; a pose names its field by index
 * (pose_field, device int32 per pose; NULL: every pose uses field 0).  At
 * most SAM_MAX_BILINEAR_FIELDS fields per call.  Poses are device float
 * arrays of 3 per pose (x, y, theta_deg).  A pose whose field index is out
 * of range or whose coordinates are not finite (or exceed 2^24 in x, y)
 * gets NaN outputs.  FP32 arithmetic with sin/cos of the pose in FP64.  All
 * calls are stream-ordered and allocation-free; they do not synchronise.
 * Errors: SAM_ERR_ARG (level, counts, null pointers, field sizes), SAM_ERR_CUDA.
 * ------------------------------------------------------------------------- */
#define SAM_MAX_BILINEAR_FIELDS 64
typedef struct {
    const float *field; /* device, FP32 (wx, wy) per pixel */
    int w, h;           /* pixels */
    int pitch;          /* row pitch in pixels, >= w */
} sam_field_ref;

/* Forward: score[b] = M_c at pose b.  Optional outputs (NULL to skip):
 * grad[3b ..] = dM_c/d(x, y, theta_deg); normal[9b ..] = the normal
 * equations of the Gauss-Newton fit of every term to 1, (1/n) sum J_i J_i^T
 * packed (xx, xy, xt, yy, yt, tt) then (1/n) sum J_i (1 - term_i), where
 * J_i = d term_i / d(x, y, theta_deg). */
sam_status sam_score_bilinear(sam_model *m, int level, const sam_field_ref *fields, int n_fields,
                              const int32_t *pose_field, const float *poses, int n_poses, float *score, float *grad,
                              float *normal, void *stream);

/* Adjoint: grad_pose[3b ..] = grad_score[b] * dM_c/d(x, y, theta_deg) at
 * pose b (the vector-Jacobian product of the forward).  grad_score and
 * grad_pose device float arrays of n_poses and 3 n_poses. */
sam_status sam_score_bilinear_adjoint(sam_model *m, int level, const sam_field_ref *fields, int n_fields,
                                      const int32_t *pose_field, const float *poses, int n_poses,
                                      const float *grad_score, float *grad_pose, void *stream);

/* Quantised-direction score map (response maps; an approximation of
 * Eq. (1), the paper has no counterpart).  Every rotated model direction is
 * replaced by the centre of its orientation bin (nbins bins over 360
 * degrees, over 180 degrees for polarity 1; bin = nearest centre, computed
 * on the host in FP64 and cached on the model), so the window maximum of
 * Eq. (1) depends only on the bin: the response maps
 *   R_b(x, y) = max over the window at (x, y) of u_b . w_hat (|.|), for
 *   -1 <= x <= w, -1 <= y <= h,
 * are computed once, then every pose of the step-1 grid is a gather-add
 *   map[(k * h + y) * w + x] = (1/n) sum_i R_{b_i(k)}(x + ox_i, y + oy_i)
 * (0 for a centre farther outside).  |map - Eq. (1)| <= 2 sin(bin width / 4).
 *   field   device FP32 pixel-layout unit field (w x h x 2 floats, 8-byte
 *           aligned), e.g. from sam_gradient.
 *   nbins   2 .. 64.
 *   maps    device scratch of sam_response_maps_bytes(w, h, nbins) bytes
 *           (holds the response maps after the call).
 *   map     device float array of num_angles(level) * h * w.
 * Two launches, stream-ordered.  The first call per (level, nbins) builds
 * the bin table on the host, allocates its device copy (cudaMalloc; held by
 * the model until sam_free_model) and uploads it on `stream`: make that
 * first call outside stream capture.  A scaled model's tables are binned per
 * table (scale and angle).  Errors: SAM_ERR_ARG, SAM_ERR_NOMEM,
 * SAM_ERR_CUDA. */
size_t sam_response_maps_bytes(int w, int h, int nbins);
sam_status sam_score_map_quantized(sam_model *m, int level, const float *field, int w, int h, int nbins,
                                   int neighbourhood, float *maps, size_t maps_bytes, float *map, void *stream);

/* Sub-pixel and sub-angle poses by a quadratic fit (extends the digitised
 * pose of Sec. II; the paper has no counterpart).  For each integer level-0
 * pose (k, y, x) -- a detection's angle_index, level0_y, level0_x -- the
 * Eq. (1) scores of the 27 poses (x + dx, y + dy, k + dk), dx, dy, dk in
 * {-1, 0, 1} (angle index circular; neighbouring search `neighbourhood`, 1
 * or 3; the model's polarity), then the stationary point of their
 * second-order Taylor model (gradient and Hessian from central differences)
 * when its Hessian is negative definite, else each axis that curves down
 * takes its own parabola's vertex and the others stay; every offset is
 * clamped to [-1/2, 1/2] (pixels, pixels, angle steps).
 *   fields, n_fields, pose_field  as sam_score_bilinear: FP32 pixel-layout
 *                    unit fields of level-0 search images; pose b uses
 *                    fields[pose_field[b]] (pose_field NULL: field 0).
 *   kyx              device int32 [n_poses][3] = (k, y, x).
 *   out              device float [n_poses][4] = (x + dx, y + dy,
 *                    theta_deg in [0, 360), M(x, y, theta_k)); NaN rows for
 *                    a pose whose field index or angle index is out of range.
 * One launch, stream-ordered, no allocation.  Errors: SAM_ERR_ARG (counts,
 * null pointers, field sizes, neighbourhood), SAM_ERR_CUDA. */
sam_status sam_subpixel_poses(sam_model *m, const sam_field_ref *fields, int n_fields, const int32_t *pose_field,
                              const int32_t *kyx, int n_poses, int neighbourhood, float *out, void *stream);

/* Sub-pixel and sub-degree refinement of n_poses poses (in place), one
 * launch: damped Gauss-Newton (Levenberg-Marquardt) on the terms of M_c,
 * each fitted to 1.  Per pose, lambda = 1e-3 and M_c with its normal
 * equations are evaluated at the start pose; then `iterations` times: solve
 * (J^T J + lambda diag(J^T J) + 1e-9 I) d = J^T r in FP64, scale d so that
 * max(|dx|, |dy|, |dtheta|) <= 1, evaluate at pose + d, and move there with
 * lambda = max(lambda/3, 1e-7) if M_c rose strictly, else lambda =
 * min(4 lambda, 1e7) (a singular system only raises lambda).  The pose is
 * carried in FP64 and written back rounded to FP32; score (device float per
 * pose, may be NULL) receives the final M_c.  0 <= iterations <= 10000. */
sam_status sam_refine_poses(sam_model *m, int level, const sam_field_ref *fields, int n_fields,
                            const int32_t *pose_field, float *poses, int n_poses, int iterations, float *score,
                            void *stream);

/* ---------------------------------------------------------------------------
 * Stage timing (tracing; the paper has no counterpart).  When enabled, sam_detect / sam_detect_batch record
 * CUDA events on the caller's stream before and after the launches of each
 * stage; sam_profile_read waits for the recorded events and adds their
 * elapsed device times to per-stage totals (so an enabled profiler adds no
 * host work between calls).  Stages: 0 pyramid, 1 gradient,
 * 2 exhaustive score map, 3 candidates, 4 refinement, 5 NMS, and within
 * stage 2: 6 the tiled scorer's launch.
 * sam_profile_read copies up to n totals (milliseconds) and call counts and
 * resets them.  Process-wide; not thread-safe.
 * ------------------------------------------------------------------------- */
#define SAM_NUM_STAGES 7
void sam_profile_enable(int on);

/* Graph mode (process-wide, on by default; the paper has no counterpart).
 * While it is on and stage timing is off, sam_detect and sam_detect_batch
 * copy the call's images into the model's workspace (one device-to-device
 * or host-to-device copy on `stream`) and replay the whole pipeline --
 * pyramid, gradients, exhaustive score, candidates, refinement, NMS -- as
 * one CUDA graph captured on the model's first call of that shape (image
 * size, batch count, detection parameters), re-captured when the shape, the
 * workspace or the scorer's tiling changes.  Results are identical to the
 * direct path, which runs while graph mode is off or stage timing is on. */
void sam_set_graph_mode(int on);
int sam_profile_read(float *ms, int *calls, int n);

/* Pose-points (the unit of the paper's Sec. II nested loops: one pose, one
 * model point) the tiled and chunked exhaustive scorers have evaluated on the
 * current device since the last reset (each warp's poses inside the map
 * times the model points it processed before finishing or being pruned by
 * early termination; without early termination this is the nominal count,
 * poses x points).  Synchronises
 * the device; reset != 0 clears the counter after reading.  -1 on a CUDA
 * error. */
long long sam_executed_pose_points(int reset);

/* Number of CUDA kernels this library has launched in this process
 * (all entry points, all devices; the paper has no counterpart).
 * Monotonic; for accounting only. */
long long sam_kernel_launches(void);

#ifdef __cplusplus
}
#endif

#endif /* SAM_H */
