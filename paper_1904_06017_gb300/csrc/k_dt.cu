// k_dt.cu -- disparity transformation (§3.3) on the device.
//
//  k_dt_moments: sums over the fitted pixels, with coordinates centred on the image
//      middle (u~ = u - (W-1)/2, v~ = v - (H-1)/2) for conditioning:
//      n, Su, Sv, Sd, Suu, Suv, Svv, Sud, Svd, Sdd -- FP32 within runs of 64 pixels
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
#include <algorithm>

#include "dt_trig.cuh"
#include "internal.cuh"

namespace sgb {

constexpr int kMom = 10;

// A thread sums runs of kRun consecutive pixels.  Inside a run every quantity is taken
// relative to the run's first fitted pixel (its column, row and disparity), so the FP32
// sums are sums of small integers and small disparity offsets -- exact or all but exact;
// each run is then shifted back to raw centred moments and added in FP64.  (The residual
// energy of the fit is a small difference of large moments, so the moments must be far
// more accurate than FP32 sums of raw values; GB300 runs FP64 at a small fraction of its
// FP32 rate, so FP64 per pixel would make this kernel FP64-bound.)  A run is read in
// pieces of kPiece pixels.
constexpr int kRun = 64, kPiece = 32;

int dt_moment_blocks(size_t n_pixels)
{
    const size_t per_block = (size_t)kDtThreads * kRun;
    const size_t nb = (n_pixels + per_block - 1) / per_block;
    return (int)std::max<size_t>(1, std::min<size_t>(nb, kDtMaxBlocks));
}

// Sum over the 32 lanes of a warp of the kMom values m[] of every lane, by a transposing
// reduction: at each of the shuffle distances 16, 8, 4, 2 a lane keeps half of its values
// (the half its lane bit selects), adds the partner's copy of that half and passes on the
// other half, so the values per lane go 16 -> 8 -> 4 -> 2 -> 1 (kMom padded to 16 with
// zeros); the last shuffle (distance 1) adds the two lanes that hold the same moment.  Each
// lane makes 16 FP64 additions instead of the 5 kMom of a butterfly on every value.  Returns
// the total of moment *k on this lane (both lanes of an even-odd pair hold the same total;
// *k >= kMom marks padding).
__device__ __forceinline__ double warp_sum_transposed(const double (&m)[kMom], int lane, int *k)
{
    static_assert(kMom <= 16, "16 slots");
    double a[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) a[i] = i < kMom ? m[i] : 0.0;
#pragma unroll
    for (int len = 8; len >= 1; len >>= 1) {   // shuffle distance 2 * len
        const bool hi = (lane & (2 * len)) != 0;
#pragma unroll
        for (int i = 0; i < len; ++i) {
            const double keep = hi ? a[len + i] : a[i];
            const double give = hi ? a[i] : a[len + i];
            a[i] = keep + __shfl_xor_sync(0xffffffffu, give, 2 * len);
        }
    }
    *k = ((lane >> 4) & 1) * 8 + ((lane >> 3) & 1) * 4 + ((lane >> 2) & 1) * 2 + ((lane >> 1) & 1);
    return a[0] + __shfl_xor_sync(0xffffffffu, a[0], 1);
}

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
    // a full piece of an aligned map is read with 16-byte loads, the rest per pixel
    const bool vec = (((uintptr_t)disp | (uintptr_t)mask) & 15) == 0;
    for (size_t run = (size_t)blockIdx.x * blockDim.x + threadIdx.x; run < nrun;
         run += (size_t)gridDim.x * blockDim.x) {
        const size_t i0 = run * kRun;
        float dref = 0.f;
        int cref = 0, rref = 0;
        bool have = false;
        float n = 0.f, su = 0.f, sv = 0.f, se = 0.f, suu = 0.f, suv = 0.f, svv = 0.f, sue = 0.f, sve = 0.f,
              see = 0.f;
        int col = (int)(i0 % W), row = (int)(i0 / W);   // one division per run
        for (int piece = 0; piece < kRun / kPiece; ++piece) {
            const size_t p0 = i0 + (size_t)piece * kPiece;
            if (p0 >= N) break;
            const int cnt = (int)min((size_t)kPiece, N - p0);
            float dv[kPiece];
            uint32_t fit = 0;   // bit j: pixel p0 + j is in the mask
            if (vec && cnt == kPiece) {
                const float4 *p4 = reinterpret_cast<const float4 *>(disp + p0);
#pragma unroll
                for (int q = 0; q < kPiece / 4; ++q) {
                    const float4 t = __ldg(p4 + q);
                    dv[4 * q] = t.x;
                    dv[4 * q + 1] = t.y;
                    dv[4 * q + 2] = t.z;
                    dv[4 * q + 3] = t.w;
                }
                if (mask) {
                    const uint4 *m4 = reinterpret_cast<const uint4 *>(mask + p0);
#pragma unroll
                    for (int q = 0; q < kPiece / 16; ++q) {
                        const uint4 t = __ldg(m4 + q);
                        const uint32_t w[4] = {t.x, t.y, t.z, t.w};
#pragma unroll
                        for (int j = 0; j < 16; ++j)
                            fit |= (uint32_t)(((w[j >> 2] >> (8 * (j & 3))) & 0xffu) != 0) << (16 * q + j);
                    }
                } else {
                    fit = 0xffffffffu;
                }
            } else {
#pragma unroll
                for (int j = 0; j < kPiece; ++j) {
                    dv[j] = 0.f;
                    if (j < cnt) {
                        dv[j] = __ldg(disp + p0 + j);
                        fit |= (uint32_t)(!mask || __ldg(mask + p0 + j) != 0) << j;
                    }
                }
            }
#pragma unroll
            for (int j = 0; j < kPiece; ++j, ++col) {
                if (col == W) {
                    col = 0;
                    ++row;
                }
                if (!((fit >> j) & 1u)) continue;
                const float d = dv[j];
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
    // the block's sums: a transposing reduction inside each warp, then the 8 warps' totals
    __shared__ double wsum[kDtThreads / 32][kMom];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int k;
    const double t = warp_sum_transposed(m, lane, &k);
    if (!(lane & 1) && k < kMom) wsum[warp][k] = t;
    __syncthreads();
    if (threadIdx.x < kMom) {
        double a = 0.0;
#pragma unroll
        for (int w = 0; w < kDtThreads / 32; ++w) a += wsum[w][threadIdx.x];
        part[(size_t)blockIdx.x * kMom + threadIdx.x] = a;
    }
}

// E and dE/dpsi per pixel at a roll psi; also alpha1 and sin / cos of psi, so that the
// accepted candidate of the search needs no second evaluation.  1/n and 2/n are taken once
// (a division per candidate would lengthen the FP64 dependency chain of every step).
struct RollModel {
    double n, inv_n, two_inv_n, Cuu, Cuv, Cvv, Cud, Cvd, Cdd;
    __device__ void eval(double psi, double *E, double *g, double *a1, double *sp, double *cp) const
    {
        double s, c;
        sincos_half_pi(psi, &s, &c);   // psi is wrapped into (-pi/2, pi/2]
        const double Cyy = c * c * Cvv - 2.0 * c * s * Cuv + s * s * Cuu;
        const double Cyd = c * Cvd - s * Cud;
        const double Cxy = (c * c - s * s) * Cuv + c * s * (Cvv - Cuu);
        const double Cxd = c * Cud + s * Cvd;
        const double al1 = Cyy > 0.0 ? Cyd / Cyy : 0.0;
        *a1 = al1;
        *sp = s;
        *cp = c;
        *E = (Cdd - al1 * Cyd) * inv_n;
        *g = al1 * (Cxd - al1 * Cxy) * two_inv_n;
    }
};

constexpr unsigned kSearchMask = 0xffffffffu;   // the 32 lanes of warp 0 evaluate candidates

// 2^-h for 0 <= h <= 1022, so that lam * pow2_neg(h) equals ldexp(lam, -h) (both are the
// exact product rounded once) without ldexp's special-case handling on the dependency chain
__device__ __forceinline__ double pow2_neg(int h)
{
    return __longlong_as_double((long long)(1023 - h) << 52);
}

// psi mapped into (-pi/2, pi/2] (E_t,min has period pi); one floor instead of an FP64 fmod
__device__ double wrap_half_pi(double psi)
{
    if (psi > 0.5 * M_PI || psi <= -0.5 * M_PI) psi -= M_PI * floor(psi * (1.0 / M_PI) + 0.5);
    if (psi > 0.5 * M_PI) psi -= M_PI;
    else if (psi <= -0.5 * M_PI) psi += M_PI;
    return psi;
}

__global__ void __launch_bounds__(kDtThreads)
k_dt_solve(const double *__restrict__ part, int nblocks, int W, int H, double psi_init, double lambda0,
           double delta_psi, int max_iters, float delta_t, stereo_dt_result *__restrict__ res,
           float *__restrict__ coef)
{
    // The partials, one moment per warp (warps 0 and 1 take a second one): lane l adds
    // partials l, l + 32, ... four loads at a time, then the warp adds its 32 lane sums with
    // a butterfly of shuffles.  (An FP64 add has a latency of about 65 cycles on GB300, and a
    // block-wide tree over all 256 threads spent most of its time adding zeros.)
    static_assert(kMom <= 2 * (kDtThreads / 32), "two moments per warp at most");
    __shared__ double tot[kMom];
    {
        const int warp = threadIdx.x >> 5, l = threadIdx.x & 31;
        const int k0 = warp, k1 = warp + kDtThreads / 32;
        double a0 = 0.0, a1 = 0.0;
        for (int b0 = l; b0 < nblocks; b0 += 128) {
            double v0[4], v1[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int b = b0 + 32 * q;
                v0[q] = (b < nblocks && k0 < kMom) ? part[(size_t)b * kMom + k0] : 0.0;
                v1[q] = (b < nblocks && k1 < kMom) ? part[(size_t)b * kMom + k1] : 0.0;
            }
            a0 += (v0[0] + v0[1]) + (v0[2] + v0[3]);
            a1 += (v1[0] + v1[1]) + (v1[2] + v1[3]);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            a0 += __shfl_xor_sync(0xffffffffu, a0, o);
            a1 += __shfl_xor_sync(0xffffffffu, a1, o);
        }
        if (l == 0 && k0 < kMom) tot[k0] = a0;
        if (l == 0 && k1 < kMom) tot[k1] = a1;
    }
    __syncthreads();
    if (threadIdx.x >= 32) return;   // warp 0 runs the search
    const int lane = threadIdx.x;
    const double n = tot[0], su = tot[1], sv = tot[2], sd = tot[3];
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
    M.inv_n = 1.0 / n;
    M.two_inv_n = 2.0 * M.inv_n;
    M.Cuu = tot[4] - su * su * M.inv_n;
    M.Cuv = tot[5] - su * sv * M.inv_n;
    M.Cvv = tot[6] - sv * sv * M.inv_n;
    M.Cud = tot[7] - su * sd * M.inv_n;
    M.Cvd = tot[8] - sv * sd * M.inv_n;
    M.Cdd = tot[9] - sd * sd * M.inv_n;

    // Every lane keeps the same search state.  A step is tried with rate lam; if the energy
    // rises the rate is halved (backtracking, at most 60 times).  The 32 lanes evaluate the
    // rates lam / 2^base, ..., lam / 2^(base + 31) at once and the lowest lane whose energy
    // does not rise wins -- the same choice as trying them one after another.
    double psi = wrap_half_pi(psi_init), lam = lambda0, E, g, a1, sn, cs;
    M.eval(psi, &E, &g, &a1, &sn, &cs);
    int status = STEREO_ENOCONV, it = 0;
    for (it = 1; it <= max_iters; ++it) {
        double step = 0.0, psi_new = psi, E_new = E, g_new = g, a1_new = a1, s_new = sn, c_new = cs;
        bool found = false;
        for (int base = 0; base < 64 && !found; base += 32) {
            const int h = base + lane;                    // halvings for this lane
            const double lam_h = lam * pow2_neg(h);
            const double st = lam_h * g;
            const double pn = wrap_half_pi(psi - st);
            double En, gn, an, sm, cm;
            M.eval(pn, &En, &gn, &an, &sm, &cm);
            const bool ok = h == 60 || (h < 60 && !(En > E));   // after 60 halvings the step stands
            const unsigned mask = __ballot_sync(kSearchMask, ok && h <= 60);
            if (mask) {
                const int src = __ffs(mask) - 1;
                step = __shfl_sync(kSearchMask, st, src);
                psi_new = __shfl_sync(kSearchMask, pn, src);
                E_new = __shfl_sync(kSearchMask, En, src);
                g_new = __shfl_sync(kSearchMask, gn, src);
                a1_new = __shfl_sync(kSearchMask, an, src);
                s_new = __shfl_sync(kSearchMask, sm, src);
                c_new = __shfl_sync(kSearchMask, cm, src);
                lam *= pow2_neg(base + src);
                found = true;
            }
        }
        const bool done = fabs(step) < delta_psi || g_new == 0.0 || g_new == g;
        const double lam_next = (g != g_new) ? lam * g / (g - g_new) : lam;   // eq. (adaptive_lambda)
        psi = psi_new;
        E = E_new;
        g = g_new;
        a1 = a1_new;
        sn = s_new;
        cs = c_new;
        if (done) {
            status = STEREO_OK;
            break;
        }
        if (isfinite(lam_next) && lam_next > 0.0) lam = lam_next;
    }
    if (lane != 0) return;
    if (it > max_iters) it = max_iters;
    // E, alpha1, sin and cos at the final psi are those of the accepted candidate
    const double s = sn, c = cs;
    const double uc = 0.5 * (W - 1), vc = 0.5 * (H - 1);
    // centred intercept, then back to raw pixel coordinates: y_raw = y~ + (vc cos - uc sin)
    const double a0c = (sd - a1 * (c * sv - s * su)) * M.inv_n;
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

// Rows whose start and the output are 16-byte aligned are done 4 pixels per thread with
// 16-byte loads and stores; the per-row term fmaf(-kc, v, k0) is the same value either way.
__global__ void k_dt_apply(const float *__restrict__ disp, int W, int H, const float *__restrict__ coef,
                           float *__restrict__ out)
{
    const int v = blockIdx.y;
    if (v >= H) return;
    const float k0 = coef[0], ks = coef[1], kc = coef[2];
    const float rowc = fmaf(-kc, (float)v, k0);
    const size_t o = (size_t)v * W;
    const bool vec = (W & 3) == 0 && (((uintptr_t)disp | (uintptr_t)out) & 15) == 0;
    if (vec) {
        const int u = 4 * (blockIdx.x * blockDim.x + threadIdx.x);
        if (u >= W) return;
        const float4 d = __ldg(reinterpret_cast<const float4 *>(disp + o + u));
        float4 r;
        r.x = d.x + fmaf(ks, (float)u, rowc);
        r.y = d.y + fmaf(ks, (float)(u + 1), rowc);
        r.z = d.z + fmaf(ks, (float)(u + 2), rowc);
        r.w = d.w + fmaf(ks, (float)(u + 3), rowc);
        *reinterpret_cast<float4 *>(out + o + u) = r;
        return;
    }
    for (int u = blockIdx.x * blockDim.x + threadIdx.x; u < W; u += gridDim.x * blockDim.x)
        out[o + u] = disp[o + u] + fmaf(ks, (float)u, rowc);
}

int launch_dt(stereo_ctx *ctx, const float *disp, const uint8_t *mask, double psi_init, float delta_t,
              float *out, stereo_dt_result *res_dev, cudaStream_t s)
{
    const Geometry &g = ctx->g;
    const size_t N = (size_t)g.W * g.H;
    const int nb = dt_moment_blocks(N);
    k_dt_moments<<<nb, kDtThreads, 0, s>>>(disp, mask, g.W, g.H, ctx->mom_part);
    int rc = cuda_error(cudaGetLastError(), "k_dt_moments launch");
    if (rc) return rc;
    k_dt_solve<<<1, kDtThreads, 0, s>>>(ctx->mom_part, nb, g.W, g.H, psi_init, ctx->p.lambda0,
                                        ctx->p.delta_psi, ctx->p.max_iters, delta_t, res_dev, ctx->dt_coef);
    rc = cuda_error(cudaGetLastError(), "k_dt_solve launch");
    if (rc) return rc;
    dim3 block(128), grid((g.W + 4 * 128 - 1) / (4 * 128), g.H);   // 4 pixels per thread where aligned
    k_dt_apply<<<grid, block, 0, s>>>(disp, g.W, g.H, ctx->dt_coef, out);
    return cuda_error(cudaGetLastError(), "k_dt_apply launch");
}

}  // namespace sgb
