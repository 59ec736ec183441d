/*
 * stereo.h -- C ABI of the GB300 (sm_103a) road-stereo library.
 *
 * The library computes the data-parallel hot path of Fan et al., "Real-Time Dense
 * Stereo Embedded in A UAV for Road Inspection" (arXiv 1904.06017):
 *   1. the perspective transformation of the target image (§3.1, eq. relation_vd),
 *   2. the matching cost c(p, d) of eq. (c),
 *   3. the bilateral aggregation of eq. (omega_s) / eq. (fbs),
 *   4. winner-take-all, the add-back of the row shift and the parabola step of
 *      eq. (subpixel) (§3.2.2),
 *   5. the disparity transformation of §3.3: roll angle (eq. e_min_gd,
 *      eq. adaptive_lambda), line fit (eq. alpha3) and the per-pixel map of
 *      eq. (disparity_transformation).
 * Steps 2-4 run in one fused kernel; the cost volume never reaches device memory.
 *
 * Conventions shared by every call:
 *   - Images are row-major uint8 (grey levels), width W, height H, row pitch in
 *     bytes (a multiple of 16, >= W).  u is the column, v the row, origin top-left.
 *   - Disparity maps are row-major float32 [H][W] (pitch W elements).
 *   - Every pointer argument named *_dev is device memory the caller owns; the
 *     library never frees or keeps it.  Host pointers are named *_host.
 *   - Calls are asynchronous on the given stream (a cudaStream_t; NULL is the
 *     legacy default stream) unless stated otherwise.
 *   - Every call returns STEREO_OK (0) or a negative STEREO_E* code and never
 *     aborts; stereo_last_error() then describes the failure (thread-local).
 *   - Numeric readings where the paper is silent (rounding of the row shift,
 *     clamp-to-edge reads, population statistics, sigma used without a factor 2,
 *     out-of-image neighbours left out, lowest d wins a tie) follow the plain
 *     definitions stated at each call.
 */
#ifndef STEREO_GB300_H
#define STEREO_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- status codes */
#define STEREO_OK 0
#define STEREO_EINVAL (-1)    /* bad argument (null pointer, size, alignment, parameter) */
#define STEREO_ENOMEM (-2)    /* device allocation failed */
#define STEREO_ECUDA (-3)     /* a CUDA runtime / driver call failed */
#define STEREO_ETIMEOUT (-4)  /* a kernel gave up a bounded wait (device status word) */
#define STEREO_ENOCONV (-5)   /* the roll search hit max_iters before |dpsi| < delta_psi */
#define STEREO_ENOTSUP (-6)   /* the configuration is not supported by the kernels */

/* cost storage type inside the fused kernel (aggregation always accumulates in FP32) */
#define STEREO_F32 0
#define STEREO_F16 1
#define STEREO_BF16 2

typedef struct CUstream_st *stereo_stream_t;   /* same type as cudaStream_t */
typedef struct stereo_ctx stereo_ctx;

/* Problem parameters, fixed for the life of a context. */
typedef struct {
    int32_t width, height;   /* W, H in pixels; 1 <= W, H <= 16384 */
    int32_t pitch;           /* bytes per image row; multiple of 16, >= width */
    int32_t max_disp;        /* D: residual disparities 0..D-1 after the warp; 1..256 */
    int32_t win;             /* NCC block size w (odd, 3..11): n = w*w in eq. (c) */
    int32_t bil;             /* bilateral window k (odd, 1..15); 11 is the paper's
                                120-connected neighbourhood (§4.4.1) */
    float sigma0, sigma1;    /* eq. (omega_s), used exactly as printed (no factor 2) */
    int32_t cost_dtype;      /* STEREO_F32 | STEREO_F16 | STEREO_BF16 */
    double lambda0;          /* initial rate of eq. (e_min_gd); paper: 10 (§4.4.2) */
    double delta_psi;        /* stop when |psi_k+1 - psi_k| < delta_psi; paper: pi/1.8e6 */
    int32_t max_iters;       /* cap on the roll iterations (default 100) */
    int32_t fused_form;      /* which kernel runs cost + aggregation + WTA (not in the paper):
                                STEREO_FUSED_AUTO (0, default), STEREO_FUSED_SIMT or
                                STEREO_FUSED_TENSOR; see below */
} stereo_params;

/* stereo_params.fused_form.  Every form computes eq. (c), eq. (fbs), the WTA and eq. (subpixel).
 *   STEREO_FUSED_SIMT    the aggregation in FP32 (or FP16 / BF16 storage with FP32 weights) on
 *                        the CUDA cores, 64 x 36 tiles, 12 disparities per chunk.
 *   STEREO_FUSED_TENSOR  FP32 storage: the screened form -- the aggregation screened on the
 *                        tensor cores with a certified error bound, the certified candidates
 *                        refined with the SIMT form's FP32 arithmetic; its outputs equal the SIMT
 *                        form's bit for bit (bil <= 13).  FP16 / BF16 storage: the tensor-core
 *                        aggregation of the 16-bit costs on the screened form's 32 x 36 tiles,
 *                        with weights rounded from the FP32 ones (bil <= 13).  (Batches may also
 *                        take 64 x 36 tiles with weights formed in 16-bit arithmetic, tile_wc 16.)
 *   STEREO_FUSED_AUTO    TENSOR where it applies, else SIMT.
 * stereo_create returns STEREO_ENOTSUP when TENSOR is asked for and does not apply. */
#define STEREO_FUSED_AUTO 0
#define STEREO_FUSED_SIMT 1
#define STEREO_FUSED_TENSOR 2

/* Result of the disparity transformation (§3.3).  alpha0 is in raw pixel
 * coordinates, so the fitted road is alpha0 + alpha1 * (v cos psi - u sin psi). */
typedef struct {
    double psi;       /* roll angle in (-pi/2, pi/2], eq. (e_min_min) */
    double alpha0;    /* eq. (alpha3) at psi */
    double alpha1;
    double e_min;     /* eq. (E_min2) at psi, summed over the fitted pixels */
    int32_t iters;    /* roll iterations taken */
    int32_t status;   /* STEREO_OK, STEREO_ENOCONV, or STEREO_EINVAL (< 2 pixels) */
    int64_t n;        /* number of fitted pixels */
} stereo_dt_result;

/* Fill *p with the defaults: sigma0 = 1.5, sigma1 = 5.5, bil = 11 (§4.4.1),
 * win = 9, lambda0 = 10, delta_psi = pi / 1.8e6 (§4.4.2), max_iters = 100,
 * cost_dtype = STEREO_F32.  Sizes are left 0 for the caller to set. */
int stereo_params_default(stereo_params *p);

/* Validate *p and create a context on the current CUDA device.  The context owns
 * padded image staging buffers, window statistics, tensor maps and the small
 * scratch of the disparity transformation (all allocated here, none later).
 * Errors: STEREO_EINVAL for bad parameters, STEREO_ENOMEM, STEREO_ECUDA. */
int stereo_create(const stereo_params *p, stereo_ctx **out);

/* Free a context and everything it owns (synchronises the device).  NULL is a no-op. */
int stereo_destroy(stereo_ctx *ctx);

/* §3.1, eq. (relation_vd): road disparity is affine in the row, du(v) = c0 + c1 v.
 * Writes the row shift s(v) = c0 + c1 v - delta_p for v = 0..height-1 to host
 * memory.  Pure host helper (no CUDA). */
int stereo_row_shift_affine(int32_t height, double c0, double c1, double delta_p,
                            float *shift_host_out);

/* §3.1: perspective transformation of the target image.  Every point of target
 * row v moves s_i(v) = floor(s(v) + 0.5) pixels to the right:
 *     tgt_warped(u, v) = tgt(clamp(u - s_i(v), 0, W-1), v).
 * tgt_dev, tgt_warped_dev: uint8 [H][pitch] (must not overlap); shift_dev: float [H].
 * Bytes u >= W of each output row are left untouched. */
int stereo_warp_target(stereo_ctx *ctx, const uint8_t *tgt_dev, const float *shift_dev,
                       uint8_t *tgt_warped_dev, stereo_stream_t stream);

/* §3.2: fused cost (eq. c) + bilateral aggregation (eq. fbs) + WTA + eq. (subpixel).
 *   c(p,d)  = 1 - NCC of the w x w reference block at p and the warped-target block
 *             at p - [d,0] (population statistics, clamp-to-edge reads; c = 1 when a
 *             block has zero variance);
 *   E(p,d)  = sum_q w(p,q) c(q,d) / sum_q w(p,q) over in-image q of the k x k window,
 *             w(p,q) = exp(-|p-q|^2/sigma0^2 - (I_ref(p) - I_ref(q))^2/sigma1^2);
 *   d*(p)   = lowest argmin_d E(p,d), d in [0, D);
 *   disp(p) = d* + delta + s_i(v), delta per eq. (subpixel) on E (0 at d* in
 *             {0, D-1} or when the denominator is not positive).
 * ref_dev, tgt_warped_dev: uint8 [H][pitch]; shift_dev: float [H] (the shift used by
 * the warp); disp_dev: float [H][W].  Optional (may be NULL): wta_dev int32 [H][W]
 * receives d*; valid_dev uint8 [H][W] receives 1 where no read behind any disparity
 * (block and bilateral window, radius m = w/2 + k/2) is clamped, in the reference,
 * the warped target, or the original target behind the warp.
 * The call launches a staging kernel (replicate padding and window statistics into
 * the context's buffers) and the fused kernel; calls on one context must not overlap. */
int stereo_cost_aggregate_wta(stereo_ctx *ctx, const uint8_t *ref_dev,
                              const uint8_t *tgt_warped_dev, const float *shift_dev,
                              float *disp_dev, int32_t *wta_dev, uint8_t *valid_dev,
                              stereo_stream_t stream);

/* stereo_cost_aggregate_wta with one more optional output: best2_dev float [H][W][2]
 * receives the normalised aggregated cost of eq. (fbs) at d* and the smallest one over
 * d != d* (their gap is a confidence of the match; with FP16 / BF16 cost storage both
 * carry that storage's rounding).  NULL skips it (the call is then stereo_cost_aggregate_wta).
 * The output comes from separate kernel instantiations, built for FP32 storage with the
 * default chunk of 12 disparities and for the tensor-core FP16 / BF16 form; a context on
 * another form (FP16 / BF16 with bil = 15 or sigma1 > 150, or FP32 windows large enough to
 * fall back to 4-disparity chunks) returns STEREO_ENOTSUP for a non-NULL best2_dev.
 * Errors: as stereo_cost_aggregate_wta, and STEREO_ENOTSUP as above. */
int stereo_cost_aggregate_wta_ex(stereo_ctx *ctx, const uint8_t *ref_dev,
                                 const uint8_t *tgt_warped_dev, const float *shift_dev,
                                 float *disp_dev, int32_t *wta_dev, uint8_t *valid_dev,
                                 float *best2_dev, stereo_stream_t stream);

/* §3.3: disparity transformation of a disparity map.
 * Fits over the pixels with mask_dev != 0 (all pixels when mask_dev is NULL) and a
 * finite disparity: 10 FP64 moments on the device, then the roll search of
 * eq. (e_min_gd) with the rate of eq. (adaptive_lambda) from psi_init, with the
 * rate applied to the energy per pixel, backtracking (a step that raises the
 * energy is halved, at most 60 times), psi wrapped into (-pi/2, pi/2], stop at
 * |dpsi| < delta_psi or max_iters; then alpha = J(psi) d (eq. alpha3) and
 *     disp_out(p) = disp(p) - alpha0 + alpha1 (u sin psi - v cos psi) + delta_t
 * (eq. disparity_transformation) for every pixel.
 * disp_dev, disp_out_dev: float [H][W] (may be the same buffer); mask_dev: uint8 [H][W].
 * res: a stereo_dt_result in device memory (the call stays asynchronous) or in
 * host memory (the call synchronises the stream and copies it back); may be NULL.
 * A non-converged search still transforms the map with the last iterate and
 * reports status STEREO_ENOCONV in res; the call itself returns STEREO_OK. */
int stereo_disparity_transform(stereo_ctx *ctx, const float *disp_dev, const uint8_t *mask_dev,
                               double psi_init, float delta_t, float *disp_out_dev,
                               stereo_dt_result *res, stereo_stream_t stream);

/* ---------------------------------------------------------- unfused reference path
 * The same arithmetic as stereo_cost_aggregate_wta, one stage per kernel, with the
 * FP32 volumes in device memory (the "plain FP32" form, and a way to inspect
 * costs and aggregated costs).  Volumes are float [H][W][D] (d fastest). */

/* eq. (c) for every pixel and d in [0, D): cost_dev float [H][W][D]. */
int stereo_cost_volume(stereo_ctx *ctx, const uint8_t *ref_dev, const uint8_t *tgt_warped_dev,
                       float *cost_dev, stereo_stream_t stream);

/* eq. (fbs) of a cost volume: agg_dev float [H][W][D] (must not alias cost_dev). */
int stereo_aggregate_volume(stereo_ctx *ctx, const uint8_t *ref_dev, const float *cost_dev,
                            float *agg_dev, stereo_stream_t stream);

/* WTA + eq. (subpixel) on an aggregated volume.  disp_dev float [H][W]; optional
 * wta_dev int32 [H][W] (d*) and best2_dev float [H][W][2] (E at d*, and the smallest
 * E over d != d*). */
int stereo_wta_volume(stereo_ctx *ctx, const float *agg_dev, const float *shift_dev,
                      float *disp_dev, int32_t *wta_dev, float *best2_dev,
                      stereo_stream_t stream);

/* ---------------------------------------------------------------- batches of pairs
 * Many stereo pairs of uneven sizes and search ranges, processed as one unit (not in the
 * paper; a throughput form of the same per-pair path).  A batch runs, for every pair, the
 * warp (§3.1), the fused cost/aggregation/WTA/sub-pixel step (§3.2) and the disparity
 * transformation (§3.3), with the fused step of all pairs in ONE persistent launch that
 * takes (pair, tile) work items heaviest first from a device counter.  The whole batch is
 * captured once into a CUDA graph at creation and replayed by stereo_batch_run.
 * The pairs' buffers are fixed at creation (the graph reads and writes them): change the
 * image contents between runs, not the pointers. */
typedef struct {
    int32_t width, height, pitch, max_disp;   /* as in stereo_params, per pair */
    const uint8_t *ref_dev;                   /* [H][pitch] reference */
    const uint8_t *tgt_dev;                   /* [H][pitch] target (warped inside the batch) */
    const float *shift_dev;                   /* [H] row shift s(v) */
    uint8_t *tgt_warped_dev;                  /* [H][pitch] scratch for the warped target */
    float *disp_dev;                          /* [H][W] disparity (output) */
    uint8_t *valid_dev;                       /* [H][W] validity mask (output; also the fit mask) */
    float *disp_out_dev;                      /* [H][W] transformed disparity (output) */
    stereo_dt_result *res_dev;                /* device result of the transformation (output) */
    double psi_init;                          /* roll search start */
    float delta_t;                            /* eq. (disparity_transformation) offset */
    int32_t *wta_dev;                         /* [H][W] integer WTA disparity d* (optional output, or NULL) */
} stereo_pair_desc;

typedef struct {
    int32_t win, bil;          /* shared by all pairs */
    float sigma0, sigma1;
    int32_t cost_dtype;        /* STEREO_F32 | STEREO_F16 | STEREO_BF16 */
    double lambda0, delta_psi;
    int32_t max_iters;
    int32_t tile_wc;           /* tile shape: warp columns 1 (32x72), 2 (64x36), 4 (128x18); 8: 64x16
                                  tiles with the costs of the next chunk computed by separate producer
                                  warps while consumer warps aggregate (FP32 storage, tile_dc 12,
                                  bil <= 11); 16: 64x36 tiles with the aggregation on the tensor cores
                                  (FP16 / BF16 storage, tile_dc 16, bil <= 13, sigma1 <= 150);
                                  32: 32x36 tiles with the aggregation on the tensor cores, 32
                                  disparities per chunk (tile_dc 32, bil <= 13; FP32 storage: the
                                  screened form, see stereo_params.fused_form); 0 = autotune */
    int32_t tile_dc;           /* disparities per chunk (12 or 4; 16 with tile_wc 16; 32 with
                                  tile_wc 32); 0 = autotune */
} stereo_batch_params;

typedef struct stereo_batch stereo_batch;

/* Defaults: the stereo_params_default values, autotuned tiles (tile_wc = tile_dc = 0). */
int stereo_batch_params_default(stereo_batch_params *p);

/* Create a batch of n pairs (pairs_host: n descriptors in host memory, copied).  With
 * tile_wc or tile_dc 0 the tile shape and chunk size are chosen by timing every candidate
 * on this batch (the candidates write into the pairs' output buffers); the choice is
 * cached in the JSON file named by the environment variable STEREO_AUTOTUNE_CACHE, keyed
 * by the pair sizes, search ranges, windows, storage type and SM count.  Allocates the
 * per-pair staging buffers and captures the CUDA graph.  Synchronous. */
int stereo_batch_create(const stereo_batch_params *p, int32_t n, const stereo_pair_desc *pairs_host,
                        stereo_batch **out);

/* Launch the batch's graph on the stream (asynchronous). */
int stereo_batch_run(stereo_batch *b, stereo_stream_t stream);

/* The tile configuration in use, the number of work items, and whether it came from the
 * autotuner cache (1), from timing (2) or from the parameters (0). */
int stereo_batch_config(const stereo_batch *b, int32_t *tile_wc, int32_t *tile_dc, int32_t *n_items,
                        int32_t *source);

/* Synchronise the device, read and clear every pair's device status word. */
int stereo_batch_check_device_status(stereo_batch *b);

/* Free the batch (synchronises the device).  NULL is a no-op. */
int stereo_batch_destroy(stereo_batch *b);

/* ---------------------------------------------------- disparity transformation, no allocation
 * The paper has no counterpart to this call: it exists for callers that cannot allocate
 * device memory (a host framework that owns the whole device heap, a real-time loop that
 * must never block in cudaMalloc, a plug-in forbidden to allocate after start-up).
 * It computes exactly what stereo_disparity_transform computes, for a width x height map,
 * with the search parameters passed directly instead of through a context, and calls no
 * cudaMalloc, cudaFree or other allocating routine.  Its scratch (partial moments of up
 * to 1024 blocks and the final coefficients, 80 KiB + 64 B) is a fixed array inside the
 * library's device image, present on every device that loads the library until exit.
 *   - The first call on each device looks up that array's device address
 *     (cudaGetSymbolAddress); make that first call before any stream capture.  The address
 *     is cached with the unique id of the context it was read in; a call in a new context
 *     (after cudaDeviceReset, say) looks it up again, so that first call in the new context
 *     also belongs before any capture.
 *   - The first call into the library in a process (this one or any other) initialises the
 *     library's CUDA runtime, which loads the library's device code: the driver takes device
 *     memory for that image then (about 16 MiB), not this call.  A caller that cannot let
 *     free memory move at all makes one call during start-up.
 *   - Every call shares the one array and leaves its last contents there; nothing in it
 *     needs to start at zero.  Calls whose kernels overlap on the GPU (other streams, other
 *     host threads) race on it: serialise them.
 *   - width, height must be 1..16384 (the same limit as stereo_create); larger maps are
 *     rejected with STEREO_EINVAL.
 * disp_dev, disp_out_dev: float [height][width]; mask_dev: uint8 or NULL; res_dev: a
 * stereo_dt_result in device memory, or NULL.  Asynchronous on the stream. */
int stereo_disparity_transform_noalloc(int32_t width, int32_t height, const float *disp_dev,
                                       const uint8_t *mask_dev, double psi_init, float delta_t,
                                       double lambda0, double delta_psi, int32_t max_iters,
                                       float *disp_out_dev, stereo_dt_result *res_dev,
                                       stereo_stream_t stream);

/* ---------------------------------------------------------------- LR-consistency check
 * §3.2.1 stores the matching costs in two volumes, one per view, and §3.2.2 removes occluded
 * reference pixels with eq. (lrc): p is dropped when
 *     (l_ref(p) - l_tar(p - [l_ref(p), 0]))^2 > delta_r        (the paper takes delta_r = 1).
 * This call computes the target view and the check for a pair whose reference view already
 * ran through stereo_cost_aggregate_wta (with a wta_dev output):
 *   - the target view matches the w x w block of the warped target around x against the
 *     reference block around x + [d, 0] (eq. c with the images exchanged, the same clamp and
 *     statistics readings), aggregates with eq. (omega_s)/(fbs) guided by the warped target,
 *     and takes the lowest d of the minimum (WTA);
 *   - both views are compared as integer WTA disparities before the sub-pixel step, in the
 *     warped target's columns: the row shift s_i(v) is added to both and cancels;
 *   - a partner column u - wta_ref(u) outside the image fails the check.
 * ref_dev, tgt_warped_dev, shift_dev: the inputs of that reference-view call; wta_ref_dev:
 * its int32 [H][W] output.  wta_tgt_dev: int32 [H][W] target-view disparities (column u of
 * the warped target), or NULL.  lr_ok_dev: uint8 [H][W], 1 where the pixel is kept.
 * delta_r: the threshold, >= 0.  Runs the fused kernel a second time, on the horizontally
 * mirrored pair with the roles of the images exchanged, which is the target view exactly;
 * it reuses the context's staging buffers.  Asynchronous on the stream.
 * Errors: STEREO_EINVAL (null pointer, negative or non-finite delta_r, a context made by a
 * batch), STEREO_ECUDA. */
int stereo_lr_check(stereo_ctx *ctx, const uint8_t *ref_dev, const uint8_t *tgt_warped_dev,
                    const float *shift_dev, const int32_t *wta_ref_dev, int32_t *wta_tgt_dev,
                    uint8_t *lr_ok_dev, float delta_r, stereo_stream_t stream);

/* ---------------------------------------------------------------- self-estimated warp model
 * The paper obtains the perspective transformation of §3.1 from correspondences it does not
 * specify; its road disparity is affine in the row, du(v) = c0 + c1 v (eq. relation_vd).
 * This object estimates c0, c1 from the unwarped pair itself, with a coarse first pass:
 *   1. both images are averaged over factor x factor blocks (the integer block sum plus
 *      factor^2/2, divided by factor^2: the mean rounded half up); a remainder of fewer than
 *      `factor` rows or columns is left out;
 *   2. the reference view (eq. c, eq. fbs, WTA, eq. subpixel) runs on the coarse pair over the
 *      full range Dc = ceil(max_disp / factor), with no warp;
 *   3. FP64 least squares over the coarse pixels the geometric validity keeps:
 *      factor * l_c(u_c, v_c) = a + b v_c, then c1 = b / factor and c0 = a - c1 (factor - 1) / 2
 *      (coarse row v_c is centred on full row factor v_c + (factor - 1) / 2).
 * max_disp: the full-resolution disparity range of the unwarped pair (1 .. 256 * factor).
 * factor: 1..8, with width / factor >= 1 and height / factor >= 1.  win, bil, sigma0, sigma1:
 * as in stereo_params, applied at the coarse resolution.  Allocates its coarse buffers and a
 * coarse context.  Errors: STEREO_EINVAL, STEREO_ENOMEM, STEREO_ECUDA, STEREO_ENOTSUP. */
typedef struct stereo_warp_est stereo_warp_est;

int stereo_warp_est_create(int32_t width, int32_t height, int32_t pitch, int32_t max_disp, int32_t factor,
                           int32_t win, int32_t bil, float sigma0, float sigma1, stereo_warp_est **out);

/* Estimate from ref_dev, tgt_dev (uint8 [height][pitch], the unwarped pair).  coef_dev:
 * double [3] in device memory = (c0, c1, n) with n the number of fitted coarse pixels; c0 and
 * c1 are NaN when fewer than two distinct coarse rows are fitted.  shift_dev: float [height]
 * receiving the row shift s(v) = c0 + c1 v - delta_p for stereo_warp_target, or NULL.
 * Asynchronous on the stream. */
int stereo_warp_est_run(stereo_warp_est *e, const uint8_t *ref_dev, const uint8_t *tgt_dev, double delta_p,
                        double *coef_dev, float *shift_dev, stereo_stream_t stream);

/* The coarse disparity map and validity of the last run (device pointers owned by the object,
 * float / uint8 [height_c][width_c], valid until it is destroyed) and their size. */
int stereo_warp_est_coarse(const stereo_warp_est *e, const float **disp_dev, const uint8_t **valid_dev,
                           int32_t *width_c, int32_t *height_c);

/* Free the object (synchronises the device).  NULL is a no-op. */
int stereo_warp_est_destroy(stereo_warp_est *e);

/* ---------------------------------------------------------------- diagnostics */

/* Synchronise the stream, read and clear the context's device status word.
 * Returns STEREO_OK, or STEREO_ETIMEOUT when a kernel gave up a bounded wait. */
int stereo_check_device_status(stereo_ctx *ctx, stereo_stream_t stream);

/* Test hook of the failure path above (no counterpart in the paper).  With on != 0, later
 * fused launches of this context (stereo_cost_aggregate_wta, _ex, stereo_lr_check) arm each
 * tile's staging barrier but issue no copy, so every CTA's bounded wait expires after about
 * a millisecond with nothing in flight; the CTA sets the status word and returns, the
 * launch's outputs are invalid, and stereo_check_device_status reports STEREO_ETIMEOUT (and
 * clears the word).  on = 0 restores normal launches; the context stays usable.  No fault,
 * trap or hang is involved.  Returns STEREO_OK, or STEREO_EINVAL for a NULL context. */
int stereo_debug_stall_staging(stereo_ctx *ctx, int32_t on);

/* Timing of the fused kernel alone: when enabled (on != 0), every later
 * stereo_cost_aggregate_wta records CUDA events on its stream around the fused
 * launch (up to 4096 launches).  stereo_profile_read synchronises and returns the
 * number of launches timed and their total milliseconds, then resets the log. */
int stereo_profile_enable(stereo_ctx *ctx, int32_t on);
int stereo_profile_read(stereo_ctx *ctx, int32_t *launches, double *total_ms);

/* FP32 FMA throughput probe (a measurement aid): runs independent chains of scalar
 * FMAs, then of packed f32x2 FMAs, on every SM (blocks_per_sm CTAs of 256 threads
 * per SM) and returns the achieved GFLOP/s of each (2 flops per FMA lane).
 * Synchronous on the legacy default stream. */
int stereo_fp32_peak_probe(int32_t blocks_per_sm, double *gflops_scalar, double *gflops_packed);

/* Description of the last error on this thread (never NULL). */
const char *stereo_last_error(void);

/* Library version string. */
const char *stereo_version(void);

#ifdef __cplusplus
}
#endif
#endif /* STEREO_GB300_H */
