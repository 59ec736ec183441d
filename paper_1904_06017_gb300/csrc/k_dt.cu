// k_dt.cu -- disparity transformation (§3.3) on the device.
//
//  k_dt_moments: sums over the fitted pixels, with coordinates centred on the image
//      middle (u~ = u - (W-1)/2, v~ = v - (H-1)/2) for conditioning:
//      n, Su, Sv, Sd, Suu, Suv, Svv, Sud, Svd, Sdd -- FP32 within runs of 32 pixels
//      (everything relative to the run's first fitted pixel), FP64 across runs, threads
//      and blocks; one partial per block.
//  k_dt_solve (one block): adds the partials in a fixed order, then one thread runs
//      the roll search.  For a roll psi, with x = u cos + v sin (eq. x) and
//      y = v cos - u sin (eq. y) and C.. the centred cross-products,
//          alpha1 = C_yd / C_yy                          (eq. alpha3)
//          E(psi) = C_dd - alpha1 C_yd                   (eq. E_min2)
//          dE/dpsi = 2 alpha1 (C_xd - alpha1 C_xy)       (eq. d_e_min with eq. M)
//      all from the ten moments.  The search (eq. e_min_gd, eq. adaptive_lambda) uses
//      E / n with backtracking, psi wrapped into (-pi/2, pi/2] (eq. e_min_min); one warp
//      evaluates 32 backtracking candidates at a time.
//  k_dt_apply: eq. (disparity_transformation) for every pixel, FP32.
#include "internal.cuh"

namespace sgb {

constexpr int kMom = 10;

// A thread sums runs of kRun consecutive pixels.  Inside a run every quantity is taken
// relative to the run's first fitted pixel (its column, row and disparity), so the FP32
// sums are sums of small integers and small disparity offsets -- exact or all but exact;
// each run is then shifted back to raw centred moments and added in FP64.  (The residual
// energy of the fit is a small difference of large moments, so the moments must be far
// more accurate than FP32 sums of raw values; GB300 runs FP64 at a small fraction of its
// FP32 rate, so FP64 per pixel would make this kernel FP64-bound.)
constexpr int kRun = 32;

__global__ void __launch_bounds__(kDtThreads)
k_dt_moments(const float *__restrict__ disp, const uint8_t *__restrict__ mask, int W, int H,
             double *__restrict__ part)
{
    double m[kMom];
#pragma unroll
    for (int k = 0; k < kMom; ++k) m[k] = 0.0;
    const double uc = 0.5 * (W - 1), vc = 0.5 * (H - 1);
    const size_t N = (size_t)W * H;
    const size_t nrun = (N + kRun - 1) / kRun;
    for (size_t run = (size_t)blockIdx.x * blockDim.x + threadIdx.x; run < nrun;
         run += (size_t)gridDim.x * blockDim.x) {
        const size_t i0 = run * kRun;
        const int cnt = (int)min((size_t)kRun, N - i0);
        float dref = 0.f;
        int cref = 0, rref = 0;
        bool have = false;
        float n = 0.f, su = 0.f, sv = 0.f, se = 0.f, suu = 0.f, suv = 0.f, svv = 0.f, sue = 0.f, sve = 0.f,
              see = 0.f;
        int col = (int)(i0 % W), row = (int)(i0 / W);   // one division per run
        for (int j = 0; j < cnt; ++j, ++col) {
            if (col == W) {
                col = 0;
                ++row;
            }
            const size_t i = i0 + j;
            if (mask && !mask[i]) continue;
            const float d = disp[i];
            if (!isfinite(d)) continue;
            if (!have) {
                dref = d;
                cref = col;
                rref = row;
                have = true;
            }
            const float u = (float)(col - cref), v = (float)(row - rref), e = d - dref;
            n += 1.f;
            su += u;
            sv += v;
            se += e;
            suu = fmaf(u, u, suu);
            suv = fmaf(u, v, suv);
            svv = fmaf(v, v, svv);
            sue = fmaf(u, e, sue);
            sve = fmaf(v, e, sve);
            see = fmaf(e, e, see);
        }
        if (!have) continue;
        // back to centred coordinates and raw disparities: x = x_local + x_ref
        const double ur = cref - uc, vr = rref - vc, dr = dref;
        const double N1 = n, Su = su, Sv = sv, Se = se;
        m[0] += N1;
        m[1] += Su + N1 * ur;
        m[2] += Sv + N1 * vr;
        m[3] += Se + N1 * dr;
        m[4] += (double)suu + 2.0 * ur * Su + N1 * ur * ur;
        m[5] += (double)suv + vr * Su + ur * Sv + N1 * ur * vr;
        m[6] += (double)svv + 2.0 * vr * Sv + N1 * vr * vr;
        m[7] += (double)sue + dr * Su + ur * Se + N1 * ur * dr;
        m[8] += (double)sve + dr * Sv + vr * Se + N1 * vr * dr;
        m[9] += (double)see + 2.0 * dr * Se + N1 * dr * dr;
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

// psi mapped into (-pi/2, pi/2] (E_t,min has period pi); one floor instead of an FP64 fmod
__device__ double wrap_half_pi(double psi)
{
    if (psi > 0.5 * M_PI || psi <= -0.5 * M_PI) psi -= M_PI * floor(psi / M_PI + 0.5);
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
    if (threadIdx.x >= 32) return;   // warp 0 runs the search, one candidate step per lane
    const int lane = threadIdx.x;
    const double n = red[0][0], su = red[1][0], sv = red[2][0], sd = red[3][0];
    stereo_dt_result r;
    r.n = (int64_t)n;
    r.iters = 0;
    if (n < 2.0) {
        if (lane != 0) return;
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

    // Every lane keeps the same search state.  A step is tried with rate lam; if the energy
    // rises the rate is halved (backtracking, at most 60 times).  The 32 lanes evaluate the
    // rates lam, lam/2, ..., lam/2^31 at once and the lowest lane whose energy does not rise
    // wins -- the same choice as trying them one after another.
    double psi = wrap_half_pi(psi_init), lam = lambda0, E, g, a1;
    M.eval(psi, &E, &g, &a1);
    int status = STEREO_ENOCONV, it = 0;
    for (it = 1; it <= max_iters; ++it) {
        double step = 0.0, psi_new = psi, E_new = E, g_new = g;
        bool found = false;
        for (int base = 0; base < 64 && !found; base += 32) {
            const int h = base + lane;                    // halvings for this lane
            const double lam_h = ldexp(lam, -h);
            const double st = lam_h * g;
            const double pn = wrap_half_pi(psi - st);
            double En, gn, an;
            M.eval(pn, &En, &gn, &an);
            const bool ok = h == 60 || (h < 60 && !(En > E));   // after 60 halvings the step stands
            const unsigned mask = __ballot_sync(0xffffffffu, ok && h <= 60);
            if (mask) {
                const int src = __ffs(mask) - 1;
                step = __shfl_sync(0xffffffffu, st, src);
                psi_new = __shfl_sync(0xffffffffu, pn, src);
                E_new = __shfl_sync(0xffffffffu, En, src);
                g_new = __shfl_sync(0xffffffffu, gn, src);
                lam = ldexp(lam, -(base + src));
                found = true;
            }
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
    if (lane != 0) return;
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
    int nb = (int)((N + (size_t)kDtThreads * kRun - 1) / ((size_t)kDtThreads * kRun));
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
