// k_dt.cu -- disparity transformation (§3.3) on the device.
//
//  k_dt_moments: FP64 sums over the fitted pixels, with coordinates centred on the
//      image middle (u~ = u - (W-1)/2, v~ = v - (H-1)/2) for conditioning:
//      n, Su, Sv, Sd, Suu, Suv, Svv, Sud, Svd, Sdd; one partial per block.
//  k_dt_solve (one block): adds the partials in a fixed order, then one thread runs
//      the roll search.  For a roll psi, with x = u cos + v sin (eq. x) and
//      y = v cos - u sin (eq. y) and C.. the centred cross-products,
//          alpha1 = C_yd / C_yy                          (eq. alpha3)
//          E(psi) = C_dd - alpha1 C_yd                   (eq. E_min2)
//          dE/dpsi = 2 alpha1 (C_xd - alpha1 C_xy)       (eq. d_e_min with eq. M)
//      all from the ten moments.  The search (eq. e_min_gd, eq. adaptive_lambda) uses
//      E / n with backtracking, psi wrapped into (-pi/2, pi/2] (eq. e_min_min).
//  k_dt_apply: eq. (disparity_transformation) for every pixel, FP32.
#include "internal.cuh"

namespace sgb {

constexpr int kMom = 10;

__global__ void __launch_bounds__(kDtThreads)
k_dt_moments(const float *__restrict__ disp, const uint8_t *__restrict__ mask, int W, int H,
             double *__restrict__ part)
{
    double m[kMom];
#pragma unroll
    for (int k = 0; k < kMom; ++k) m[k] = 0.0;
    const double uc = 0.5 * (W - 1), vc = 0.5 * (H - 1);
    const size_t N = (size_t)W * H;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (size_t)gridDim.x * blockDim.x) {
        if (mask && !mask[i]) continue;
        const float df = disp[i];
        if (!isfinite(df)) continue;
        const double d = df;
        const double u = (double)(i % W) - uc, v = (double)(i / W) - vc;
        m[0] += 1.0;
        m[1] += u;
        m[2] += v;
        m[3] += d;
        m[4] += u * u;
        m[5] += u * v;
        m[6] += v * v;
        m[7] += u * d;
        m[8] += v * d;
        m[9] += d * d;
    }
    __shared__ double red[kMom][kDtThreads];
#pragma unroll
    for (int k = 0; k < kMom; ++k) red[k][threadIdx.x] = m[k];
    __syncthreads();
    for (int s = kDtThreads / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s)
#pragma unroll
            for (int k = 0; k < kMom; ++k) red[k][threadIdx.x] += red[k][threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x < kMom) part[(size_t)blockIdx.x * kMom + threadIdx.x] = red[threadIdx.x][0];
}

struct RollModel {
    double n, Cuu, Cuv, Cvv, Cud, Cvd, Cdd;
    __device__ void eval(double psi, double *E, double *g, double *a1) const
    {
        double s, c;
        sincos(psi, &s, &c);
        const double Cyy = c * c * Cvv - 2.0 * c * s * Cuv + s * s * Cuu;
        const double Cyd = c * Cvd - s * Cud;
        const double Cxy = (c * c - s * s) * Cuv + c * s * (Cvv - Cuu);
        const double Cxd = c * Cud + s * Cvd;
        const double al1 = Cyy > 0.0 ? Cyd / Cyy : 0.0;
        *a1 = al1;
        *E = (Cdd - al1 * Cyd) / n;
        *g = 2.0 * al1 * (Cxd - al1 * Cxy) / n;
    }
};

__device__ double wrap_half_pi(double psi)
{
    psi = fmod(psi, M_PI);
    if (psi > 0.5 * M_PI) psi -= M_PI;
    else if (psi <= -0.5 * M_PI) psi += M_PI;
    return psi;
}

__global__ void __launch_bounds__(kDtThreads)
k_dt_solve(const double *__restrict__ part, int nblocks, int W, int H, double psi_init, double lambda0,
           double delta_psi, int max_iters, float delta_t, stereo_dt_result *__restrict__ res,
           float *__restrict__ coef)
{
    __shared__ double red[kMom][kDtThreads];
    double m[kMom];
#pragma unroll
    for (int k = 0; k < kMom; ++k) m[k] = 0.0;
    for (int b = threadIdx.x; b < nblocks; b += kDtThreads)
#pragma unroll
        for (int k = 0; k < kMom; ++k) m[k] += part[(size_t)b * kMom + k];
#pragma unroll
    for (int k = 0; k < kMom; ++k) red[k][threadIdx.x] = m[k];
    __syncthreads();
    for (int s = kDtThreads / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s)
#pragma unroll
            for (int k = 0; k < kMom; ++k) red[k][threadIdx.x] += red[k][threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x != 0) return;
    const double n = red[0][0], su = red[1][0], sv = red[2][0], sd = red[3][0];
    stereo_dt_result r;
    r.n = (int64_t)n;
    r.iters = 0;
    if (n < 2.0) {
        r.psi = 0.0;
        r.alpha0 = n > 0 ? sd / n : 0.0;
        r.alpha1 = 0.0;
        r.e_min = 0.0;
        r.status = STEREO_EINVAL;
        *res = r;
        coef[0] = (float)(-r.alpha0 + delta_t);
        coef[1] = 0.f;
        coef[2] = 0.f;
        return;
    }
    RollModel M;
    M.n = n;
    M.Cuu = red[4][0] - su * su / n;
    M.Cuv = red[5][0] - su * sv / n;
    M.Cvv = red[6][0] - sv * sv / n;
    M.Cud = red[7][0] - su * sd / n;
    M.Cvd = red[8][0] - sv * sd / n;
    M.Cdd = red[9][0] - sd * sd / n;

    double psi = wrap_half_pi(psi_init), lam = lambda0, E, g, a1;
    M.eval(psi, &E, &g, &a1);
    int status = STEREO_ENOCONV, it = 0;
    for (it = 1; it <= max_iters; ++it) {
        double step = lam * g;
        double psi_new = wrap_half_pi(psi - step), E_new, g_new, a1n;
        M.eval(psi_new, &E_new, &g_new, &a1n);
        for (int h = 0; h < 60 && E_new > E; ++h) {   // backtracking
            lam *= 0.5;
            step = lam * g;
            psi_new = wrap_half_pi(psi - step);
            M.eval(psi_new, &E_new, &g_new, &a1n);
        }
        const bool done = fabs(step) < delta_psi || g_new == 0.0 || g_new == g;
        const double lam_next = (g != g_new) ? lam * g / (g - g_new) : lam;   // eq. (adaptive_lambda)
        psi = psi_new;
        E = E_new;
        g = g_new;
        if (done) {
            status = STEREO_OK;
            break;
        }
        if (isfinite(lam_next) && lam_next > 0.0) lam = lam_next;
    }
    if (it > max_iters) it = max_iters;
    M.eval(psi, &E, &g, &a1);
    double s, c;
    sincos(psi, &s, &c);
    const double uc = 0.5 * (W - 1), vc = 0.5 * (H - 1);
    // centred intercept, then back to raw pixel coordinates: y_raw = y~ + (vc cos - uc sin)
    const double a0c = (sd - a1 * (c * sv - s * su)) / n;
    const double a0 = a0c - a1 * (vc * c - uc * s);
    r.psi = psi;
    r.alpha0 = a0;
    r.alpha1 = a1;
    r.e_min = E * n;
    r.iters = it;
    r.status = status;
    *res = r;
    // l' = l - alpha0 + alpha1 sin(psi) u - alpha1 cos(psi) v + delta_t
    coef[0] = (float)(-a0 + (double)delta_t);
    coef[1] = (float)(a1 * s);
    coef[2] = (float)(a1 * c);
}

__global__ void k_dt_apply(const float *__restrict__ disp, int W, int H, const float *__restrict__ coef,
                           float *__restrict__ out)
{
    const int u = blockIdx.x * blockDim.x + threadIdx.x, v = blockIdx.y;
    if (u >= W || v >= H) return;
    const float k0 = coef[0], ks = coef[1], kc = coef[2];
    const size_t o = (size_t)v * W + u;
    out[o] = disp[o] + fmaf(ks, (float)u, fmaf(-kc, (float)v, k0));
}

int launch_dt(stereo_ctx *ctx, const float *disp, const uint8_t *mask, double psi_init, float delta_t,
              float *out, stereo_dt_result *res_dev, cudaStream_t s)
{
    const Geometry &g = ctx->g;
    const size_t N = (size_t)g.W * g.H;
    int nb = (int)((N + (size_t)kDtThreads * 8 - 1) / ((size_t)kDtThreads * 8));
    if (nb > kDtMaxBlocks) nb = kDtMaxBlocks;
    if (nb < 1) nb = 1;
    k_dt_moments<<<nb, kDtThreads, 0, s>>>(disp, mask, g.W, g.H, ctx->mom_part);
    int rc = cuda_error(cudaGetLastError(), "k_dt_moments launch");
    if (rc) return rc;
    k_dt_solve<<<1, kDtThreads, 0, s>>>(ctx->mom_part, nb, g.W, g.H, psi_init, ctx->p.lambda0,
                                        ctx->p.delta_psi, ctx->p.max_iters, delta_t, res_dev, ctx->dt_coef);
    rc = cuda_error(cudaGetLastError(), "k_dt_solve launch");
    if (rc) return rc;
    dim3 block(128), grid((g.W + 127) / 128, g.H);
    k_dt_apply<<<grid, block, 0, s>>>(disp, g.W, g.H, ctx->dt_coef, out);
    return cuda_error(cudaGetLastError(), "k_dt_apply launch");
}

}  // namespace sgb
