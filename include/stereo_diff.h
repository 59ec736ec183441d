/*
 * stereo_diff.h -- differentiable form of the stereo path (C ABI, sm_103a).
 *
 * The paper selects the disparity by winner-take-all (§3.2.2) and differentiates only the
 * disparity-transformation energy, and only with respect to the roll angle (eq. d_e_min).
 * These calls make the whole path differentiable by replacing the hard argmin with a
 * soft-argmin at temperature T:
 *
 *   c(q,d) = 1 - NCC of the w x w blocks (eq. c) on FLOAT images, clamp-to-edge reads,
 *            population statistics; c = 1 where sigma_ref * sigma_tgt = 0
 *   E(p,d) = sum_q w(p,q) c(q,d) / sum_q w(p,q)        (eq. omega_s, eq. fbs; out-of-image q
 *            left out; sigma0, sigma1 used as printed, without a factor 2)
 *   l(p)   = sum_d d softmax_d(-E(p,d) / T) + s_i(v)   (s_i = floor(s(v) + 0.5), §3.1; with
 *            STEREO_WARP_LINEAR the fractional s(v) itself, the target read by interpolation)
 *   L      = sum_p m(p) (l(p) - alpha0 - alpha1 y_p(psi))^2,  y_p = v cos(psi) - u sin(psi)
 *            (eq. E2, eq. y; raw pixel coordinates, u the column, v the row)
 *
 * The target enters through the row-shift warp of §3.1, so gradients reach the unwarped
 * target image.  All arithmetic is FP32 except the energy reductions, which accumulate in
 * FP64.  The aggregated volume E is never stored: the backward pass recomputes it tile by
 * tile from the stored cost volume.  Reductions are in a fixed order: every call is
 * deterministic.
 *
 * Conventions (as in stereo.h): *_dev pointers are caller-owned device memory; calls are
 * asynchronous on the stream; every call returns STEREO_OK or a negative STEREO_E* code and
 * stereo_last_error() describes the failure.  A batch holds `batch` pairs of one size,
 * stored back to back: images float32 [batch][height][width] (pitch = width elements),
 * shift tables float32 [batch][height], disparities float32 [batch][height][width].
 */
#ifndef STEREO_GB300_DIFF_H
#define STEREO_GB300_DIFF_H

#include <stddef.h>
#include <stdint.h>

#include "stereo.h"

#ifdef __cplusplus
extern "C" {
#endif

/* How the target row is shifted by s(v) (§3.1). */
#define STEREO_WARP_ROUND 0   /* s_i = floor(s + 0.5), the pixel copied; s_i is added back */
#define STEREO_WARP_LINEAR 1  /* the point u - s(v) read by linear interpolation between the two
                                 neighbouring columns (each clamped to the edge); s(v) itself,
                                 unrounded, is added back -- l is then differentiable in s(v) */

typedef struct {
    int32_t width, height;   /* 1 <= W, H <= 8192 */
    int32_t batch;           /* pairs per call, 1..64 */
    int32_t max_disp;        /* D: residual disparities 0..D-1, 1..256 */
    int32_t win;             /* NCC block w, odd, 1..15 */
    int32_t bil;             /* bilateral window k, odd, 1..15 */
    float sigma0, sigma1;    /* eq. (omega_s) */
    float temperature;       /* T > 0 of the soft-argmin */
    int32_t warp_mode;       /* STEREO_WARP_ROUND (default) or STEREO_WARP_LINEAR */
} stereo_diff_params;

/* Defaults: win = 9, bil = 11, sigma0 = 1.5, sigma1 = 5.5 (§4.4.1), temperature = 0.1,
 * batch = 1, warp_mode = STEREO_WARP_ROUND; sizes and max_disp left 0 for the caller to set. */
int stereo_diff_params_default(stereo_diff_params *p);

/* Bytes of device workspace the soft-argmin forward and backward need for *p (the
 * forward writes the cost volume, window statistics and soft-max normalisers there;
 * the backward reads them and adds its own adjoint volumes).  Host only.
 * Errors: STEREO_EINVAL for bad parameters. */
int stereo_softargmin_workspace_bytes(const stereo_diff_params *p, size_t *bytes);

/* Forward: disp_dev = l for every pair (see the definition above).  ref_dev, tgt_dev:
 * float32 images; shift_dev: the row-shift tables.  workspace_dev: at least the bytes
 * reported above, 256-byte aligned; its contents after this call are what
 * stereo_softargmin_bwd needs, so keep it untouched between the two.
 * Errors: STEREO_EINVAL (null pointer, bad parameters, small or unaligned workspace),
 * STEREO_ECUDA. */
int stereo_softargmin_fwd(const stereo_diff_params *p, const float *ref_dev, const float *tgt_dev,
                          const float *shift_dev, float *disp_dev, void *workspace_dev,
                          size_t workspace_bytes, stereo_stream_t stream);

/* Backward (vector-Jacobian product): given grad_disp_dev = dS/dl for a scalar S, write
 * grad_ref_dev = dS/dref and grad_tgt_dev = dS/dtgt (float32 [batch][height][width]) and
 * grad_shift_dev = dS/ds(v) (float32 [batch][height]), overwritten, not accumulated.
 * ref_dev, tgt_dev, shift_dev and the workspace must be those of the matching forward call.
 * Any of the three outputs may be NULL to skip it.  The cost adjoint of eq. (c) is taken
 * with the statistics of each window pair; a pair with sigma_ref * sigma_tgt = 0 (c fixed at
 * 1) passes no gradient.  With STEREO_WARP_ROUND the shift enters only through its rounding,
 * so dS/ds = 0; with STEREO_WARP_LINEAR it is the derivative of the interpolation (taken
 * inside the interval between two columns) plus that of the add-back.
 * Errors: as the forward. */
int stereo_softargmin_bwd(const stereo_diff_params *p, const float *ref_dev, const float *tgt_dev,
                          const float *shift_dev, const float *grad_disp_dev, float *grad_ref_dev,
                          float *grad_tgt_dev, float *grad_shift_dev, void *workspace_dev,
                          size_t workspace_bytes, stereo_stream_t stream);

/* Bytes of device workspace the energy calls below need for `batch` pairs (partial sums
 * of 64 blocks per pair and the refinement state).  Host only. */
int stereo_dt_energy_workspace_bytes(int32_t batch, size_t *bytes);

/* eq. (E2) per pair: energy_dev[b] = sum_p m(p) (l(p) - alpha0 - alpha1 y_p(psi))^2 with
 * theta_dev[b] = (psi, alpha0, alpha1) (float64 [batch][3], device).  disp_dev: float32
 * [batch][height][width]; mask_dev: uint8 of the same shape, nonzero = fitted, or NULL
 * for every pixel.  energy_dev: float64 [batch].  Errors: STEREO_EINVAL, STEREO_ECUDA. */
int stereo_dt_energy_fwd(int32_t width, int32_t height, int32_t batch, const float *disp_dev,
                         const uint8_t *mask_dev, const double *theta_dev, double *energy_dev,
                         void *workspace_dev, size_t workspace_bytes, stereo_stream_t stream);

/* Adjoint of eq. (E2) for upstream gradients grad_energy_dev (float64 [batch]):
 *   grad_disp_dev[b] = 2 g m r,  r = l - alpha0 - alpha1 y      (float32, or NULL to skip)
 *   grad_theta_dev[b] = (2 g alpha1 sum m r x,  -2 g sum m r,  -2 g sum m r y)
 * with x = u cos(psi) + v sin(psi) (eq. x), float64 [batch][3] or NULL to skip. */
int stereo_dt_energy_bwd(int32_t width, int32_t height, int32_t batch, const float *disp_dev,
                         const uint8_t *mask_dev, const double *theta_dev,
                         const double *grad_energy_dev, float *grad_disp_dev,
                         double *grad_theta_dev, void *workspace_dev, size_t workspace_bytes,
                         stereo_stream_t stream);

/* Roll refinement by gradient: `steps` steps of descent on psi, per pair, from psi_init.
 * At every step the line fit is re-solved, (alpha0, alpha1) = eq. (alpha3) at psi (FP64
 * normal equations), so dL/dpsi there is the gradient of eq. (E_min2) (eq. d_e_min);
 * psi moves by -g / H, H = 2 alpha1^2 |x~|^2 the Gauss-Newton curvature (x~ = x(psi)
 * with its least-squares projection on [1, y(psi)] removed), and is wrapped into
 * (-pi/2, pi/2].  A step with H <= 0 (fewer than 2 distinct fitted points) leaves psi
 * unchanged.  traj_dev: float64 [batch][steps + 1][5], entry k = (psi_k, alpha0_k,
 * alpha1_k, g_k, E_k) with E_k the energy at (psi_k, alpha(psi_k)); the last entry is
 * the result.  0 <= steps <= 1000.  Errors: STEREO_EINVAL, STEREO_ECUDA. */
int stereo_dt_refine_roll(int32_t width, int32_t height, int32_t batch, const float *disp_dev,
                          const uint8_t *mask_dev, double psi_init, int32_t steps, double *traj_dev,
                          void *workspace_dev, size_t workspace_bytes, stereo_stream_t stream);

#ifdef __cplusplus
}
#endif
#endif /* STEREO_GB300_DIFF_H */
