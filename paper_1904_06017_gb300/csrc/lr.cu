// lr.cu -- the target view and the LR-consistency check of eq. (lrc) (§3.2.1, §3.2.2).
//
// The target view matches the warped target's block around x against the reference block
// around x + [d, 0], guided by the warped target.  Mirroring both images horizontally and
// exchanging their roles turns that into the reference view of the mirrored pair: the
// mirrored target's pixel W-1-x at disparity d reads the mirrored reference at W-1-x-d, i.e.
// the reference at x + d; clamp-to-edge reads and the bilateral window are symmetric under
// the mirror.  So the fused kernel runs once more on the mirrored pair, and k_lr_check maps
// its WTA output back and applies eq. (lrc).
#include <math.h>

#include "internal.cuh"

namespace sgb {
namespace {

// out[v][W-1-u] = in[v][u] for the W image columns of every row.
__global__ void __launch_bounds__(256) k_mirror(const uint8_t *__restrict__ in, uint8_t *__restrict__ out, int W,
                                                int pitch)
{
    const int u = blockIdx.x * blockDim.x + threadIdx.x, v = blockIdx.y;
    if (u < W) out[(size_t)v * pitch + (W - 1 - u)] = in[(size_t)v * pitch + u];
}

// wta_tgt(u) = mirrored-run WTA at W-1-u; ok(u) = partner x = u - wta_ref(u) inside the image
// and (wta_ref(u) - wta_tgt(x))^2 <= delta_r.
__global__ void __launch_bounds__(256) k_lr_check(const int32_t *__restrict__ wref, const int32_t *__restrict__ wmir,
                                                  int32_t *__restrict__ wtgt, uint8_t *__restrict__ ok, int W,
                                                  float delta_r)
{
    const int u = blockIdx.x * blockDim.x + threadIdx.x, v = blockIdx.y;
    if (u >= W) return;
    const size_t row = (size_t)v * W;
    if (wtgt) wtgt[row + u] = wmir[row + (W - 1 - u)];
    const int dr = wref[row + u], x = u - dr;
    bool pass = false;
    if (x >= 0 && x < W) {
        const float diff = (float)(dr - wmir[row + (W - 1 - x)]);
        pass = diff * diff <= delta_r;
    }
    ok[row + u] = (uint8_t)pass;
}

}  // namespace
}  // namespace sgb

using namespace sgb;

extern "C" int stereo_lr_check(stereo_ctx *ctx, const uint8_t *ref, const uint8_t *tgtw, const float *shift,
                               const int32_t *wta_ref, int32_t *wta_tgt, uint8_t *lr_ok, float delta_r,
                               stereo_stream_t stream)
{
    if (!ctx || !ref || !tgtw || !shift || !wta_ref || !lr_ok)
        return set_error(STEREO_EINVAL, "stereo_lr_check: null pointer");
    if (!(delta_r >= 0.f) || !isfinite(delta_r))
        return set_error(STEREO_EINVAL, "stereo_lr_check: delta_r must be finite and >= 0");
    if (!ctx->lr_ref) return set_error(STEREO_EINVAL, "stereo_lr_check: context has no LR buffers");
    cudaStream_t s = (cudaStream_t)stream;
    const int W = ctx->p.width, H = ctx->p.height, pitch = ctx->p.pitch;
    const dim3 grid((W + 255) / 256, H);
    // the mirrored pair: the warped target becomes the reference, the reference the target
    k_mirror<<<grid, 256, 0, s>>>(tgtw, ctx->lr_ref, W, pitch);
    k_mirror<<<grid, 256, 0, s>>>(ref, ctx->lr_tgt, W, pitch);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_error(e, "stereo_lr_check: mirror");
    int rc = launch_prep(ctx, ctx->lr_ref, ctx->lr_tgt, s);
    if (!rc) rc = launch_row_tables(ctx, shift, ctx->lr_tgt, s);
    if (!rc) rc = launch_fused(ctx, shift, ctx->lr_disp, ctx->lr_wta, nullptr, s);
    if (rc) return rc;
    k_lr_check<<<grid, 256, 0, s>>>(wta_ref, ctx->lr_wta, wta_tgt, lr_ok, W, delta_r);
    return cuda_error(cudaGetLastError(), "stereo_lr_check");
}
