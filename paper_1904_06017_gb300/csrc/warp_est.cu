// warp_est.cu -- the self-estimated warp model: coarse full-range stereo and the
// least-squares line of eq. (relation_vd), du(v) = c0 + c1 v (see include/stereo.h).
#include <math.h>
#include <string.h>

#include <new>

#include "internal.cuh"

struct stereo_warp_est {
    int W, H, pitch, F, Wc, Hc, pitch_c, Dc;
    stereo_ctx *cc;            // context of the coarse pair
    uint8_t *ref_c, *tgt_c;    // block averages [Hc][pitch_c]
    float *zero_shift;         // [Hc] zeros: the coarse pass has no warp
    float *disp_c;             // [Hc][Wc]
    uint8_t *valid_c;          // [Hc][Wc]
    double *part;              // [kFitBlocks][5] partial sums
};

namespace sgb {
namespace {

constexpr int kFitBlocks = 64;

// out(uc, vc) = (sum of the F x F block + F^2 / 2) / F^2, integers.
__global__ void __launch_bounds__(256) k_block_mean(const uint8_t *__restrict__ in, int pitch, uint8_t *__restrict__ out,
                                                    int pitch_c, int Wc, int F)
{
    const int uc = blockIdx.x * blockDim.x + threadIdx.x, vc = blockIdx.y;
    if (uc >= Wc) return;
    int s = 0;
    for (int i = 0; i < F; ++i) {
        const uint8_t *row = in + (size_t)(vc * F + i) * pitch + uc * F;
        for (int j = 0; j < F; ++j) s += row[j];
    }
    out[(size_t)vc * pitch_c + uc] = (uint8_t)((s + (F * F) / 2) / (F * F));
}

// FP64 sums over the valid coarse pixels of n, v, v^2, d, v d with d = F * l_c.
__global__ void __launch_bounds__(256) k_fit_partials(const float *__restrict__ disp, const uint8_t *__restrict__ valid,
                                                      int Wc, int Hc, int F, double *__restrict__ part)
{
    __shared__ double red[8][5];
    double acc[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    const int n = Wc * Hc;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        if (!valid[i]) continue;
        const double v = (double)(i / Wc), d = (double)F * (double)disp[i];
        acc[0] += 1.0;
        acc[1] += v;
        acc[2] = fma(v, v, acc[2]);
        acc[3] += d;
        acc[4] = fma(v, d, acc[4]);
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        double x = acc[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
        if (lane == 0) red[w][k] = x;
    }
    __syncthreads();
    if (threadIdx.x < 5) {
        double x = 0.0;
        for (int j = 0; j < 8; ++j) x += red[j][threadIdx.x];
        part[blockIdx.x * 5 + threadIdx.x] = x;
    }
}

// Thread 0 adds the partials in block order and solves the 2 x 2 normal equations; then the
// block writes s(v) = c0 + c1 v - delta_p.
__global__ void __launch_bounds__(256) k_fit_finish(const double *__restrict__ part, int F, double delta_p,
                                                    double *__restrict__ coef, float *__restrict__ shift, int H)
{
    __shared__ double c[2];
    if (threadIdx.x == 0) {
        double S[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
        for (int j = 0; j < kFitBlocks; ++j)
            for (int k = 0; k < 5; ++k) S[k] += part[j * 5 + k];
        const double det = S[0] * S[2] - S[1] * S[1];
        double c0 = nan(""), c1 = nan("");
        if (S[0] >= 2.0 && det > 0.0) {
            const double a = (S[2] * S[3] - S[1] * S[4]) / det, b = (S[0] * S[4] - S[1] * S[3]) / det;
            c1 = b / F;
            c0 = a - c1 * (F - 1) * 0.5;
        }
        coef[0] = c0;
        coef[1] = c1;
        coef[2] = S[0];
        c[0] = c0;
        c[1] = c1;
    }
    __syncthreads();
    if (shift)
        for (int v = threadIdx.x; v < H; v += blockDim.x) shift[v] = (float)(c[0] + c[1] * (double)v - delta_p);
}

void free_est(stereo_warp_est *e)
{
    if (!e) return;
    if (e->cc) stereo_destroy(e->cc);
    cudaFree(e->ref_c);
    cudaFree(e->tgt_c);
    cudaFree(e->zero_shift);
    cudaFree(e->disp_c);
    cudaFree(e->valid_c);
    cudaFree(e->part);
    delete e;
}

}  // namespace
}  // namespace sgb

using namespace sgb;

extern "C" int stereo_warp_est_create(int32_t W, int32_t H, int32_t pitch, int32_t max_disp, int32_t F,
                                      int32_t win, int32_t bil, float sigma0, float sigma1, stereo_warp_est **out)
{
    static const char *who = "stereo_warp_est_create";
    if (!out) return set_error(STEREO_EINVAL, "%s: null output", who);
    *out = nullptr;
    if (F < 1 || F > 8) return set_error(STEREO_EINVAL, "%s: factor %d outside 1..8", who, F);
    if (W < F || H < F || W > kMaxDim || H > kMaxDim || pitch < W)
        return set_error(STEREO_EINVAL, "%s: size %dx%d (pitch %d) too small for factor %d", who, W, H, pitch, F);
    if (max_disp < 1 || max_disp > kMaxD * F)
        return set_error(STEREO_EINVAL, "%s: max_disp %d outside 1..%d", who, max_disp, kMaxD * F);
    stereo_warp_est *e = new (std::nothrow) stereo_warp_est();
    if (!e) return set_error(STEREO_ENOMEM, "%s: host allocation failed", who);
    memset(e, 0, sizeof(*e));
    e->W = W;
    e->H = H;
    e->pitch = pitch;
    e->F = F;
    e->Wc = W / F;
    e->Hc = H / F;
    e->pitch_c = (e->Wc + 15) / 16 * 16;
    e->Dc = (max_disp + F - 1) / F;
    stereo_params p;
    stereo_params_default(&p);
    p.width = e->Wc;
    p.height = e->Hc;
    p.pitch = e->pitch_c;
    p.max_disp = e->Dc;
    p.win = win;
    p.bil = bil;
    p.sigma0 = sigma0;
    p.sigma1 = sigma1;
    int rc = create_context(&p, 0, 0, &e->cc);
    const size_t img = (size_t)e->Hc * e->pitch_c, map = (size_t)e->Hc * e->Wc;
    if (rc || (rc = cuda_error(cudaMalloc(&e->ref_c, img), "cudaMalloc coarse ref")) ||
        (rc = cuda_error(cudaMalloc(&e->tgt_c, img), "cudaMalloc coarse tgt")) ||
        (rc = cuda_error(cudaMalloc(&e->zero_shift, sizeof(float) * e->Hc), "cudaMalloc coarse shift")) ||
        (rc = cuda_error(cudaMalloc(&e->disp_c, sizeof(float) * map), "cudaMalloc coarse disparity")) ||
        (rc = cuda_error(cudaMalloc(&e->valid_c, map), "cudaMalloc coarse validity")) ||
        (rc = cuda_error(cudaMalloc(&e->part, sizeof(double) * 5 * kFitBlocks), "cudaMalloc fit partials")) ||
        (rc = cuda_error(cudaMemset(e->zero_shift, 0, sizeof(float) * e->Hc), "cudaMemset")) ||
        (rc = cuda_error(cudaMemset(e->ref_c, 0, img), "cudaMemset")) ||
        (rc = cuda_error(cudaMemset(e->tgt_c, 0, img), "cudaMemset"))) {
        free_est(e);
        return rc;
    }
    *out = e;
    return STEREO_OK;
}

extern "C" int stereo_warp_est_run(stereo_warp_est *e, const uint8_t *ref, const uint8_t *tgt, double delta_p,
                                   double *coef, float *shift, stereo_stream_t stream)
{
    static const char *who = "stereo_warp_est_run";
    if (!e || !ref || !tgt || !coef) return set_error(STEREO_EINVAL, "%s: null pointer", who);
    if (!isfinite(delta_p)) return set_error(STEREO_EINVAL, "%s: delta_p not finite", who);
    cudaStream_t s = (cudaStream_t)stream;
    const dim3 grid((e->Wc + 255) / 256, e->Hc);
    k_block_mean<<<grid, 256, 0, s>>>(ref, e->pitch, e->ref_c, e->pitch_c, e->Wc, e->F);
    k_block_mean<<<grid, 256, 0, s>>>(tgt, e->pitch, e->tgt_c, e->pitch_c, e->Wc, e->F);
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess) return cuda_error(err, who);
    int rc = launch_prep(e->cc, e->ref_c, e->tgt_c, s);
    if (!rc) rc = launch_row_tables(e->cc, e->zero_shift, e->tgt_c, s);
    if (!rc) rc = launch_fused(e->cc, e->zero_shift, e->disp_c, nullptr, e->valid_c, s);
    if (rc) return rc;
    k_fit_partials<<<kFitBlocks, 256, 0, s>>>(e->disp_c, e->valid_c, e->Wc, e->Hc, e->F, e->part);
    k_fit_finish<<<1, 256, 0, s>>>(e->part, e->F, delta_p, coef, shift, e->H);
    return cuda_error(cudaGetLastError(), who);
}

extern "C" int stereo_warp_est_coarse(const stereo_warp_est *e, const float **disp, const uint8_t **valid,
                                      int32_t *wc, int32_t *hc)
{
    if (!e || !disp || !valid || !wc || !hc) return set_error(STEREO_EINVAL, "stereo_warp_est_coarse: null pointer");
    *disp = e->disp_c;
    *valid = e->valid_c;
    *wc = e->Wc;
    *hc = e->Hc;
    return STEREO_OK;
}

extern "C" int stereo_warp_est_destroy(stereo_warp_est *e)
{
    if (!e) return STEREO_OK;
    cudaDeviceSynchronize();
    free_est(e);
    return STEREO_OK;
}
