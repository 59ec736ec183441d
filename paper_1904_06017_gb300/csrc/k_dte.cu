// k_dte.cu -- the disparity-transformation energy of eq. (E2), its adjoint, and roll
// refinement by gradient (include/stereo_diff.h).
//
// Every reduction runs in two fixed-order stages: kDteBlocks blocks per pair write FP64
// partial sums, one finishing thread per pair adds them in index order.  Per pixel the
// energy and its adjoint work in FP32 with FP64 accumulation.  The refinement reduces the
// map once to ten FP64 moments in centred coordinates; every step then evaluates the sums it
// needs at its angle from them (exact algebra) and solves the normal equations of eq. (alpha3)
// in FP64.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "internal.cuh"
#include "stereo_diff.h"

namespace sgb {
namespace {

constexpr int kDteBlocks = 64;     // partial-sum blocks per pair
constexpr int kDteSums = 10;       // the most sums one pass produces (the refinement)
constexpr int kDteThreads = 256;

enum { DTE_ENERGY = 0, DTE_BWD = 1 };

size_t dte_bytes(int B)
{
    const size_t part = (size_t)B * kDteBlocks * kDteSums * sizeof(double);
    const size_t state = (size_t)B * 2 * sizeof(double);
    return (part + 255) / 256 * 256 + (state + 255) / 256 * 256;
}

template <int NS>
__device__ void block_sum_store(double (&acc)[NS], double *out)
{
    __shared__ double red[kDteThreads / 32][NS];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < NS; ++k) {
        double v = acc[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) red[wid][k] = v;
    }
    __syncthreads();
    if (threadIdx.x < NS) {
        double v = 0.0;
        for (int w = 0; w < kDteThreads / 32; ++w) v += red[w][threadIdx.x];
        out[threadIdx.x] = v;
    }
}

// Per pixel r = l - alpha0 - alpha1 y(psi), y = v cos(psi) - u sin(psi) (eq. y).
// DTE_ENERGY: sum m r^2.  DTE_BWD: gl = 2 g m r, sums of m r x, m r, m r y.
template <int MODE>
__global__ void __launch_bounds__(kDteThreads) k_dte(const float *__restrict__ disp, const uint8_t *__restrict__ mask,
                                                     const double *__restrict__ theta, const double *__restrict__ gE,
                                                     float *__restrict__ gdisp, double *__restrict__ part, int W,
                                                     int H)
{
    constexpr int NS = MODE == DTE_ENERGY ? 1 : 3;
    __shared__ float sc[5];
    const int b = blockIdx.y;
    if (threadIdx.x == 0) {
        const double psi = theta[3 * b];
        sc[0] = (float)cos(psi);
        sc[1] = (float)sin(psi);
        sc[2] = (float)theta[3 * b + 1];
        sc[3] = (float)theta[3 * b + 2];
        sc[4] = MODE == DTE_BWD ? (float)(2.0 * gE[b]) : 0.f;
    }
    __syncthreads();
    const float c = sc[0], s = sc[1], a0 = sc[2], a1 = sc[3], g2 = sc[4];
    const int HW = W * H;
    const float *L = disp + (size_t)b * HW;
    const uint8_t *M = mask ? mask + (size_t)b * HW : nullptr;
    double acc[NS];
#pragma unroll
    for (int k = 0; k < NS; ++k) acc[k] = 0.0;
    for (int i = blockIdx.x * kDteThreads + threadIdx.x; i < HW; i += kDteBlocks * kDteThreads) {
        const int v = i / W, u = i - v * W;
        const float m = (!M || M[i]) ? 1.f : 0.f;
        const float y = (float)v * c - (float)u * s;
        const float r = m * (L[i] - a0 - a1 * y);
        if constexpr (MODE == DTE_ENERGY) {
            acc[0] += (double)(r * r);
        } else {
            if (gdisp) gdisp[(size_t)b * HW + i] = g2 * r;
            const float x = (float)u * c + (float)v * s;
            acc[0] += (double)(r * x);
            acc[1] += (double)r;
            acc[2] += (double)(r * y);
        }
    }
    block_sum_store<NS>(acc, part + ((size_t)b * kDteBlocks + blockIdx.x) * kDteSums);
}

// One thread per pair adds the partials in block order.
template <int MODE>
__global__ void k_dte_finish(const double *__restrict__ part, const double *__restrict__ theta,
                             const double *__restrict__ gE, double *__restrict__ out, int B)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    constexpr int NS = MODE == DTE_ENERGY ? 1 : 3;
    double s[NS];
#pragma unroll
    for (int k = 0; k < NS; ++k) s[k] = 0.0;
    for (int j = 0; j < kDteBlocks; ++j)
#pragma unroll
        for (int k = 0; k < NS; ++k) s[k] += part[((size_t)b * kDteBlocks + j) * kDteSums + k];
    if constexpr (MODE == DTE_ENERGY) {
        out[b] = s[0];
    } else {
        const double g = gE[b], a1 = theta[3 * b + 2];
        out[3 * b + 0] = 2.0 * g * a1 * s[0];      // dL/dpsi: dy/dpsi = -x
        out[3 * b + 1] = -2.0 * g * s[1];          // dL/dalpha0
        out[3 * b + 2] = -2.0 * g * s[2];          // dL/dalpha1
    }
}

// The ten moments of the fitted pixels in coordinates centred on the image, FP64:
// n, S_u, S_v, S_l, S_uu, S_uv, S_vv, S_ul, S_vl, S_ll with u' = u - (W-1)/2, v' = v - (H-1)/2.
// Every sum the refinement needs at an angle psi is a fixed combination of them.
__global__ void __launch_bounds__(kDteThreads) k_dref_moments(const float *__restrict__ disp,
                                                              const uint8_t *__restrict__ mask,
                                                              double *__restrict__ part, int W, int H)
{
    const int b = blockIdx.y;
    const int HW = W * H;
    const float *L = disp + (size_t)b * HW;
    const uint8_t *M = mask ? mask + (size_t)b * HW : nullptr;
    const double uc = 0.5 * (W - 1), vc = 0.5 * (H - 1);
    double acc[kDteSums];
#pragma unroll
    for (int k = 0; k < kDteSums; ++k) acc[k] = 0.0;
    for (int i = blockIdx.x * kDteThreads + threadIdx.x; i < HW; i += kDteBlocks * kDteThreads) {
        if (M && !M[i]) continue;
        const int v = i / W, u = i - v * W;
        const double x = (double)u - uc, y = (double)v - vc, l = (double)L[i];
        acc[0] += 1.0;
        acc[1] += x;
        acc[2] += y;
        acc[3] += l;
        acc[4] = fma(x, x, acc[4]);
        acc[5] = fma(x, y, acc[5]);
        acc[6] = fma(y, y, acc[6]);
        acc[7] = fma(x, l, acc[7]);
        acc[8] = fma(y, l, acc[8]);
        acc[9] = fma(l, l, acc[9]);
    }
    block_sum_store<kDteSums>(acc, part + ((size_t)b * kDteBlocks + blockIdx.x) * kDteSums);
}

__device__ double wrap_half_pi_d(double psi)
{
    psi = fmod(psi, M_PI);
    if (psi > 0.5 * M_PI) psi -= M_PI;
    else if (psi <= -0.5 * M_PI) psi += M_PI;
    return psi;
}

// All refinement steps of one pair (one thread per pair).  At each angle the sums over the
// fitted pixels of y, y^2, l y, x, x y, x^2, l x (raw coordinates, x = u cos + v sin, y = v cos
// - u sin, eq. x, eq. y) follow from the centred moments; then the line fit of eq. (alpha3)
// from the FP64 normal equations, E and g = dE/dpsi there (eq. d_e_min), the Gauss-Newton
// curvature and the step psi <- wrap(psi - g / H).  Trajectory entry k is written at each step.
__global__ void k_dref_run(const double *__restrict__ part, const double *__restrict__ state, double *__restrict__ traj,
                           int steps, int W, int H, int B)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    double m[kDteSums];
    for (int q = 0; q < kDteSums; ++q) m[q] = 0.0;
    for (int j = 0; j < kDteBlocks; ++j)
        for (int q = 0; q < kDteSums; ++q) m[q] += part[((size_t)b * kDteBlocks + j) * kDteSums + q];
    const double n = m[0], Su = m[1], Sv = m[2], Sl = m[3], Suu = m[4], Suv = m[5], Svv = m[6], Sul = m[7],
                 Svl = m[8], Sll = m[9];
    const double uc = 0.5 * (W - 1), vc = 0.5 * (H - 1);
    double psi = state[2 * b];
    for (int k = 0; k <= steps; ++k) {
        const double c = cos(psi), s = sin(psi);
        // raw x = x' + xc, y = y' + yc with the centred rotated coordinates x', y'
        const double xc = uc * c + vc * s, yc = vc * c - uc * s;
        const double Sx1 = Su * c + Sv * s, Sy1 = Sv * c - Su * s;                // sums of x', y'
        const double Sxx1 = c * c * Suu + 2.0 * c * s * Suv + s * s * Svv;
        const double Syy1 = c * c * Svv - 2.0 * c * s * Suv + s * s * Suu;
        const double Sxy1 = c * s * (Svv - Suu) + (c * c - s * s) * Suv;
        const double Slx1 = Sul * c + Svl * s, Sly1 = Svl * c - Sul * s;
        const double Sy = Sy1 + n * yc, Sx = Sx1 + n * xc;
        const double Syy = Syy1 + 2.0 * yc * Sy1 + n * yc * yc;
        const double Sxx = Sxx1 + 2.0 * xc * Sx1 + n * xc * xc;
        const double Sxy = Sxy1 + xc * Sy1 + yc * Sx1 + n * xc * yc;
        const double Sly = Sly1 + yc * Sl, Slx = Slx1 + xc * Sl;
        const double det = n * Syy - Sy * Sy;
        double a0 = 0.0, a1 = 0.0, g = 0.0, Hc = 0.0;
        if (n > 0.0 && det > 0.0) {
            a0 = (Syy * Sl - Sy * Sly) / det;
            a1 = (n * Sly - Sy * Sl) / det;
            g = 2.0 * a1 * (Slx - a0 * Sx - a1 * Sxy);
            const double xt2 = Sxx - (Syy * Sx * Sx - 2.0 * Sy * Sx * Sxy + n * Sxy * Sxy) / det;
            Hc = 2.0 * a1 * a1 * xt2;
        } else if (n > 0.0) {
            a0 = Sl / n;
        }
        const double E = Sll - 2.0 * a0 * Sl - 2.0 * a1 * Sly + a0 * a0 * n + 2.0 * a0 * a1 * Sy + a1 * a1 * Syy;
        double *t = traj + ((size_t)b * (steps + 1) + k) * 5;
        t[0] = psi;
        t[1] = a0;
        t[2] = a1;
        t[3] = g;
        t[4] = E;
        if (k < steps && Hc > 0.0 && isfinite(g / Hc)) psi = wrap_half_pi_d(psi - g / Hc);
    }
}

__global__ void k_dref_init(double *state, double psi, int B)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b < B) {
        state[2 * b] = wrap_half_pi_d(psi);
        state[2 * b + 1] = 0.0;
    }
}

int check_sizes(int W, int H, int B, const char *who)
{
    if (W < 1 || H < 1 || W > 8192 || H > 8192)
        return set_error(STEREO_EINVAL, "%s: width/height %d x %d outside 1..8192", who, W, H);
    if (B < 1 || B > 64) return set_error(STEREO_EINVAL, "%s: batch %d outside 1..64", who, B);
    return STEREO_OK;
}

int check_dte_ws(int B, void *ws, size_t bytes, const char *who)
{
    if (!ws) return set_error(STEREO_EINVAL, "%s: null workspace", who);
    if ((uintptr_t)ws % 256) return set_error(STEREO_EINVAL, "%s: workspace not 256-byte aligned", who);
    if (bytes < dte_bytes(B))
        return set_error(STEREO_EINVAL, "%s: workspace of %zu bytes, %zu needed", who, bytes, dte_bytes(B));
    return STEREO_OK;
}

double *dte_state(int B, void *ws)
{
    const size_t part = (size_t)B * kDteBlocks * kDteSums * sizeof(double);
    return (double *)((char *)ws + (part + 255) / 256 * 256);
}

}  // namespace
}  // namespace sgb

using namespace sgb;

extern "C" int stereo_dt_energy_workspace_bytes(int32_t batch, size_t *bytes)
{
    if (batch < 1 || batch > 64 || !bytes)
        return set_error(STEREO_EINVAL, "stereo_dt_energy_workspace_bytes: batch outside 1..64 or null output");
    *bytes = dte_bytes(batch);
    return STEREO_OK;
}

extern "C" int stereo_dt_energy_fwd(int32_t W, int32_t H, int32_t B, const float *disp, const uint8_t *mask,
                                    const double *theta, double *energy, void *ws, size_t ws_bytes,
                                    stereo_stream_t stream)
{
    static const char *who = "stereo_dt_energy_fwd";
    int rc = check_sizes(W, H, B, who);
    if (rc) return rc;
    if (!disp || !theta || !energy) return set_error(STEREO_EINVAL, "%s: null pointer", who);
    if ((rc = check_dte_ws(B, ws, ws_bytes, who))) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    double *part = (double *)ws;
    k_dte<DTE_ENERGY><<<dim3(kDteBlocks, B), kDteThreads, 0, st>>>(disp, mask, theta, nullptr, nullptr, part,
                                                                    W, H);
    k_dte_finish<DTE_ENERGY><<<(B + 63) / 64, 64, 0, st>>>(part, theta, nullptr, energy, B);
    return cuda_error(cudaGetLastError(), who);
}

extern "C" int stereo_dt_energy_bwd(int32_t W, int32_t H, int32_t B, const float *disp, const uint8_t *mask,
                                    const double *theta, const double *gE, float *gdisp, double *gtheta,
                                    void *ws, size_t ws_bytes, stereo_stream_t stream)
{
    static const char *who = "stereo_dt_energy_bwd";
    int rc = check_sizes(W, H, B, who);
    if (rc) return rc;
    if (!disp || !theta || !gE) return set_error(STEREO_EINVAL, "%s: null pointer", who);
    if ((rc = check_dte_ws(B, ws, ws_bytes, who))) return rc;
    if (!gdisp && !gtheta) return STEREO_OK;
    cudaStream_t st = (cudaStream_t)stream;
    double *part = (double *)ws;
    k_dte<DTE_BWD><<<dim3(kDteBlocks, B), kDteThreads, 0, st>>>(disp, mask, theta, gE, gdisp, part, W, H);
    if (gtheta) k_dte_finish<DTE_BWD><<<(B + 63) / 64, 64, 0, st>>>(part, theta, gE, gtheta, B);
    return cuda_error(cudaGetLastError(), who);
}

extern "C" int stereo_dt_refine_roll(int32_t W, int32_t H, int32_t B, const float *disp, const uint8_t *mask,
                                     double psi_init, int32_t steps, double *traj, void *ws, size_t ws_bytes,
                                     stereo_stream_t stream)
{
    static const char *who = "stereo_dt_refine_roll";
    int rc = check_sizes(W, H, B, who);
    if (rc) return rc;
    if (!disp || !traj) return set_error(STEREO_EINVAL, "%s: null pointer", who);
    if (steps < 0 || steps > 1000) return set_error(STEREO_EINVAL, "%s: steps %d outside 0..1000", who, steps);
    if (!isfinite(psi_init)) return set_error(STEREO_EINVAL, "%s: psi_init not finite", who);
    if ((rc = check_dte_ws(B, ws, ws_bytes, who))) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    double *part = (double *)ws, *state = dte_state(B, ws);
    k_dref_init<<<(B + 63) / 64, 64, 0, st>>>(state, psi_init, B);
    k_dref_moments<<<dim3(kDteBlocks, B), kDteThreads, 0, st>>>(disp, mask, part, W, H);
    k_dref_run<<<(B + 63) / 64, 64, 0, st>>>(part, state, traj, steps, W, H, B);
    return cuda_error(cudaGetLastError(), who);
}
