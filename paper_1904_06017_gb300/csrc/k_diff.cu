// k_diff.cu -- soft-argmin disparity over the bilateral-aggregated cost and its adjoint
// (include/stereo_diff.h).  FP32 throughout; the aggregated volume E(p,d) of eq. (fbs) is
// never stored: the backward pass recomputes it tile by tile from the stored cost volume.
//
// Forward (per pair of a batch, float images):
//   k_dwarp     tw(u,v) = tgt(clamp(u - s_i(v)), v)                                   §3.1
//   k_dstats    window mean / population std of ref (image grid) and of tw (columns
//               shifted by -(D-1), so that the target window of (p, d) is the entry at u-d)
//   k_dcost     c(p,d) = 1 - sum_i (a_i - mu_a)(b_i - mu_b) / (n s_a s_b)           eq. (c)
//   k_dagg<FWD> E(p,d) = sum_q w c / sum_q w (eq. omega_s, eq. fbs), online soft-max over d:
//               l = sum_d d P(p,d) + s_i(v), P = softmax_d(-E/T); keeps log2-sum-exp, lbar
// Backward, given gl = dS/dl:
//   k_dagg<H>   recompute E; gE = -gl P (d - lbar) / T; h = gE / Z(p);  beta(p) = sum_d h E;
//               t1(p) = sum_d h(p,d) sum_q w (I_q - I_p) c(q,d) - beta(p) sum_q w (I_q - I_p)
//   k_dagg<GC>  gc(q,d) = sum_p w(p,q) h(p,d)                  (adjoint of eq. fbs in c)
//               gw(x) = 2/sigma1^2 (t1(x) + sum_d c(x,d) sum_q w (I_q - I_x) h(q,d)
//                                        - sum_q w (I_q - I_x) beta(q))  (through the weights)
//   k_dcost_bwd adjoint of eq. (c): with A = -gc/(n s_a s_b), B = gc ncc/(n s_a^2),
//               C = gc ncc/(n s_b^2) per window pair, every extended reference position X
//               collects  sum_d sum_q A (t - mu_b) + B (r - mu_a)            -> gref_ext(X)
//               and for the target position X - d:  sum_q A (r - mu_a) + C (t - mu_b) -> Gamma(X,d),
//               summed over d per X - d inside each tile (partial diagonal sums; Gamma itself
//               is never stored)
//   k_dtgt_diag gtw_ext(Xt) = sum_d Gamma(Xt + d, d): the tiles' partial sums added
//   k_dfold     fold the clamp-to-edge positions back onto the image and undo the warp
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <type_traits>

#include "internal.cuh"
#include "row_shift.cuh"
#include "stereo_diff.h"

namespace sgb {
namespace {


enum { AGG_FWD = 0, AGG_H = 1, AGG_GC = 2 };
// pixels per thread in k_dagg (a column segment): the forward pass, with one accumulator set,
// takes 8, so that each staged neighbour row serves twice the weights
__host__ __device__ constexpr int agg_rows(int mode) { return mode == AGG_FWD ? 8 : 4; }

// k_dagg tiles: the recomputing backward pass (AGG_H) double-buffers its disparity chunks on
// 64 x 24 tiles of 12 warps (one block per SM); the other two stream each chunk into one
// buffer on 32 x 32 tiles of 8 warps, several blocks per SM hiding the copies instead.
__host__ __device__ constexpr bool agg_dbuf(int mode) { return mode == AGG_H; }
__host__ __device__ constexpr int agg_tx(int mode) { return agg_dbuf(mode) ? 64 : 32; }
__host__ __device__ constexpr int agg_ty(int mode) { return agg_dbuf(mode) ? 24 : 32; }
__host__ __device__ constexpr int agg_threads(int mode)
{
    return agg_dbuf(mode) ? 384 : 32 * (agg_tx(mode) / 32) * agg_ty(mode) / agg_rows(mode);
}
constexpr int kAggDC = 8;            // disparities per chunk in k_dagg
constexpr int kCostDC = 16;          // disparities per block in k_dcost
constexpr float kFar = 1e18f;        // scaled intensity of an out-of-image neighbour: weight 0
constexpr float kLog2e = 1.4426950408889634f;

// The cost adjoint's tiles are 32 extended columns wide; each sums Gamma(X, d) over d into
// 32 + D - 1 entries per row, one per target column X - d its columns reach.
__host__ __device__ constexpr int cb_tiles_x(int Wr) { return (Wr + 31) / 32; }
__host__ __device__ constexpr int cb_diag_w(int D) { return 32 + D - 1; }

__device__ __forceinline__ int clampi(int x, int lo, int hi) { return min(max(x, lo), hi); }

// 2^x on the MUFU unit (relative error about 2^-22; -inf and huge negative x give +0).
__device__ __forceinline__ float ex2_fast(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float lane(const float2 &v, int k) { return (k & 1) ? v.y : v.x; }

// §3.1 integer row shift floor(s + 0.5) (exact for every float s), as the value added back to
// the disparity.
__device__ __forceinline__ float row_shift_value(float s) { return round_half_up(s); }

// The same shift as a column offset, limited to +-2W: every column then clamps to the same
// edge as it would with the exact value.
__device__ __forceinline__ int row_shift(float s, int W)
{
    const float lim = 2.0f * (float)W;
    return (int)fminf(fmaxf(row_shift_value(s), -lim), lim);
}

// ------------------------------------------------------------------ layout of the workspace
struct Dims {
    int W, H, B, D, rw, rb, n, warp_mode;
    int We;            // W + D - 1: target statistics columns (u - d + D - 1)
    int Wr, Hr;        // W + 2rw, H + 2rw: extended reference grid of the cost adjoint
    int Wt;            // W + 2rw + D - 1: extended target columns
};

struct Ws {
    float *tw, *mur, *sdr, *mut, *isdt, *cost, *lse, *lbar;      // forward (isdt: 1 / s_b, 0 where flat)
    float *h, *gc, *beta, *t1, *gw, *gpart, *grefx, *gtwx;      // backward
};

size_t layout(const Dims &d, char *base, Ws *w)
{
    size_t off = 0;
    auto take = [&](float **p, size_t elems) {
        if (p) *p = base ? (float *)(base + off) : nullptr;
        off += (elems * sizeof(float) + 255) / 256 * 256;
    };
    const size_t B = d.B, img = (size_t)d.H * d.W, vol = (size_t)d.D * img;
    Ws tmp;
    Ws *o = w ? w : &tmp;
    take(&o->tw, B * img);
    take(&o->mur, B * img);
    take(&o->sdr, B * img);
    take(&o->mut, B * (size_t)d.H * d.We);
    take(&o->isdt, B * (size_t)d.H * d.We);
    take(&o->cost, B * vol);
    take(&o->lse, B * img);
    take(&o->lbar, B * img);
    take(&o->h, B * vol);
    take(&o->gc, B * vol);
    take(&o->beta, B * img);
    take(&o->t1, B * img);
    take(&o->gw, B * img);
    take(&o->gpart, B * (size_t)d.Hr * cb_tiles_x(d.Wr) * cb_diag_w(d.D));
    take(&o->grefx, B * (size_t)d.Hr * d.Wr);
    take(&o->gtwx, B * (size_t)d.Hr * d.Wt);
    return off;
}

int check_params(const stereo_diff_params *p, Dims *d, const char *who)
{
    if (!p) return set_error(STEREO_EINVAL, "%s: null parameters", who);
    if (p->width < 1 || p->height < 1 || p->width > 8192 || p->height > 8192)
        return set_error(STEREO_EINVAL, "%s: width/height %d x %d outside 1..8192", who, p->width,
                         p->height);
    if (p->batch < 1 || p->batch > 64)
        return set_error(STEREO_EINVAL, "%s: batch %d outside 1..64", who, p->batch);
    if (p->max_disp < 1 || p->max_disp > 256)
        return set_error(STEREO_EINVAL, "%s: max_disp %d outside 1..256", who, p->max_disp);
    if (p->win < 1 || p->win > 15 || !(p->win & 1))
        return set_error(STEREO_EINVAL, "%s: win %d must be odd, 1..15", who, p->win);
    if (p->bil < 1 || p->bil > 15 || !(p->bil & 1))
        return set_error(STEREO_EINVAL, "%s: bil %d must be odd, 1..15", who, p->bil);
    if (!(p->sigma0 > 0.f) || !(p->sigma1 > 0.f) || !isfinite(p->sigma0) || !isfinite(p->sigma1))
        return set_error(STEREO_EINVAL, "%s: sigma0, sigma1 must be positive and finite", who);
    if (!(p->temperature > 0.f) || !isfinite(p->temperature))
        return set_error(STEREO_EINVAL, "%s: temperature must be positive and finite", who);
    if (p->warp_mode != STEREO_WARP_ROUND && p->warp_mode != STEREO_WARP_LINEAR)
        return set_error(STEREO_EINVAL, "%s: warp_mode %d unknown", who, p->warp_mode);
    d->W = p->width;
    d->H = p->height;
    d->B = p->batch;
    d->D = p->max_disp;
    d->rw = p->win / 2;
    d->rb = p->bil / 2;
    d->n = p->win * p->win;
    d->warp_mode = p->warp_mode;
    d->We = d->W + d->D - 1;
    d->Wr = d->W + 2 * d->rw;
    d->Hr = d->H + 2 * d->rw;
    d->Wt = d->W + 2 * d->rw + d->D - 1;
    return STEREO_OK;
}

int check_ws(const Dims &d, void *ws, size_t bytes, Ws *w, const char *who)
{
    const size_t need = layout(d, nullptr, nullptr);
    if (!ws) return set_error(STEREO_EINVAL, "%s: null workspace", who);
    if ((uintptr_t)ws % 256) return set_error(STEREO_EINVAL, "%s: workspace not 256-byte aligned", who);
    if (bytes < need)
        return set_error(STEREO_EINVAL, "%s: workspace of %zu bytes, %zu needed", who, bytes, need);
    layout(d, (char *)ws, w);
    return STEREO_OK;
}

// ------------------------------------------------------------------ forward kernels
// The linear-interpolation warp reads u - s = u + k + f with k = floor(-s) and f in [0, 1):
// both neighbours are the columns u + k and u + k + 1 of every pixel of the row.  k is
// limited to +-2W, where both neighbours clamp to the same edge pixel whatever f is.
struct LinShift {
    int k;
    float f;
};

__device__ __forceinline__ LinShift lin_shift(float s, int W)
{
    const float ns = -s, fl = floorf(ns), lim = 2.0f * (float)W;
    LinShift r;
    r.k = (int)fminf(fmaxf(fl, -lim), lim);
    r.f = ns - fl;
    return r;
}

__global__ void __launch_bounds__(256) k_dwarp(const float *__restrict__ tgt, const float *__restrict__ shift,
                                               float *__restrict__ tw, int W, int H, int mode)
{
    const int u = blockIdx.x * blockDim.x + threadIdx.x, v = blockIdx.y, b = blockIdx.z;
    if (u >= W) return;
    const size_t row = ((size_t)b * H + v) * W;
    const float s = shift[(size_t)b * H + v];
    if (mode == STEREO_WARP_LINEAR) {
        const LinShift ls = lin_shift(s, W);
        const float A = tgt[row + clampi(u + ls.k, 0, W - 1)], B = tgt[row + clampi(u + ls.k + 1, 0, W - 1)];
        tw[row + u] = fmaf(ls.f, B - A, A);
        return;
    }
    tw[row + u] = tgt[row + clampi(u - row_shift(s, W), 0, W - 1)];
}

// Window mean and population standard deviation over (2rw+1)^2 clamp-to-edge reads, on an
// output grid of Wout columns whose column xo is centred on image column xo + off (sd and its
// reciprocal isd are each written when their pointer is not null).
template <int RW>
__global__ void __launch_bounds__(256) k_dstats(const float *__restrict__ img, int W, int H, int Wout, int off,
                                                float *__restrict__ mu, float *__restrict__ sd,
                                                float *__restrict__ isd)
{
    extern __shared__ float s[];
    constexpr int rw = RW, sw = 32 + 2 * RW, sh = 8 + 2 * RW, w = 2 * RW + 1;
    const int x0 = blockIdx.x * 32, y0 = blockIdx.y * 8, b = blockIdx.z;
    const float *im = img + (size_t)b * H * W;
    {
        // every load of a thread before its first store
        constexpr int NI = (sw * sh + 255) / 256;
        float vi[NI];
#pragma unroll
        for (int it = 0; it < NI; ++it) {
            const int i = threadIdx.x + 256 * it, r = i / sw, c = i - r * sw;
            vi[it] = i < sw * sh ? im[(size_t)clampi(y0 - rw + r, 0, H - 1) * W + clampi(x0 + off - rw + c, 0, W - 1)]
                                 : 0.f;
        }
#pragma unroll
        for (int it = 0; it < NI; ++it) {
            const int i = threadIdx.x + 256 * it;
            if (i < sw * sh) s[i] = vi[it];
        }
    }
    __syncthreads();
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const int xo = x0 + tx, v = y0 + ty;
    if (xo >= Wout || v >= H) return;
    const float n = (float)(w * w);
    // relative to the centre value: a block whose values are all equal gets sd = 0 exactly
    const float *blk = s + ty * sw + tx;
    const float c0 = blk[rw * sw + rw];
    float sum = 0.f;
#pragma unroll 1
    for (int dy = 0; dy < w; ++dy)
#pragma unroll
        for (int dx = 0; dx < w; ++dx) sum += blk[dy * sw + dx] - c0;
    const float m = sum / n;
    float q = 0.f;
#pragma unroll 1
    for (int dy = 0; dy < w; ++dy)
#pragma unroll
        for (int dx = 0; dx < w; ++dx) {
            const float a = (blk[dy * sw + dx] - c0) - m;
            q = fmaf(a, a, q);
        }
    const size_t o = ((size_t)b * H + v) * Wout + xo;
    mu[o] = c0 + m;
    const float sv = sqrtf(q / n);
    if (sd) sd[o] = sv;
    if (isd) isd[o] = sv > 0.f ? __frcp_rn(sv) : 0.f;   // the cost adjoint's 1 / s_b, once per position
}

void launch_dstats(int rw, dim3 grid, size_t smem, cudaStream_t st, const float *img, int W, int H, int Wout, int off,
                   float *mu, float *sd, float *isd)
{
    switch (rw) {
#define SGB_DSTATS(R)                                                                  \
    case R: k_dstats<R><<<grid, 256, smem, st>>>(img, W, H, Wout, off, mu, sd, isd); break;
    SGB_DSTATS(0) SGB_DSTATS(1) SGB_DSTATS(2) SGB_DSTATS(3) SGB_DSTATS(4) SGB_DSTATS(5) SGB_DSTATS(6)
    default: k_dstats<7><<<grid, 256, smem, st>>>(img, W, H, Wout, off, mu, sd, isd); break;
#undef SGB_DSTATS
    }
}

// eq. (c) for a 64 x 8 pixel tile and kCostDC disparities: the centred reference window
// times the target window, corrected by the target mean through sum_i (a_i - mu_a).  Thread
// (tx, ty) owns the four pixels (x0 + tx + 32 j, y0 + 2 ty + h), j, h in {0, 1}, the columns
// j = 0, 1 as the two lanes of packed f32x2 operations: both images are staged as pairs
// (value at column c, value at column c + 32), so a warp's pair loads are consecutive 8-byte
// words.  Along an image row the target pairs of the DC disparities slide by one column per
// step and are kept in a register window that takes one new load per step; each image row of
// the tile's halo serves both pixel rows of the thread (window rows dy and dy - 1).  Every
// pixel and disparity takes the same terms in the same order (dy, then dx) as a scalar loop.
constexpr int kCostTX = 64, kCostTY = 8, kCostThreads = 16 * kCostTY;
__host__ __device__ constexpr int dcost_rw_pairs(int rw) { return 32 + 2 * rw; }
__host__ __device__ constexpr int dcost_tw_pairs(int rw) { return 32 + 2 * rw + kCostDC - 1; }
__host__ __device__ constexpr int dcost_rows(int rw) { return kCostTY + 2 * rw; }
constexpr int kCostSW = kCostTX + kCostDC - 1;   // target statistics per tile row
__host__ __device__ constexpr size_t dcost_smem(int rw)
{
    return (size_t)(dcost_rw_pairs(rw) + dcost_tw_pairs(rw)) * dcost_rows(rw) * sizeof(float2) +
           (size_t)2 * kCostTY * kCostSW * sizeof(float);
}

template <int RW>
__global__ void __launch_bounds__(kCostThreads, 3) k_dcost(const float *__restrict__ ref, const float *__restrict__ tw,
                                                  const float *__restrict__ mur, const float *__restrict__ sdr,
                                                  const float *__restrict__ mut, const float *__restrict__ isdt,
                                                  float *__restrict__ cost, int W, int H, int D, int nchunk)
{
    constexpr int DC = kCostDC, rw = RW, w = 2 * RW + 1;
    constexpr int PRW = dcost_rw_pairs(RW), PTW = dcost_tw_pairs(RW), SH = dcost_rows(RW);
    extern __shared__ float2 s2[];
    float2 *pr = s2, *pt = s2 + SH * PRW;        // [SH][PRW], [SH][PTW]
    float *smb = reinterpret_cast<float *>(pt + SH * PTW), *ssb = smb + kCostTY * kCostSW;   // [TY][SW]
    const int b = blockIdx.z / nchunk, d0 = (blockIdx.z % nchunk) * DC;
    const int x0 = blockIdx.x * kCostTX, y0 = blockIdx.y * kCostTY;
    const size_t HW = (size_t)H * W;
    const float *R = ref + b * HW, *T = tw + b * HW;
    // Staging: every load of a thread is issued before its first shared-memory store, so the
    // loads are in flight together rather than one L2 round trip per entry.
    const int tc0 = x0 - d0 - (DC - 1) - rw;     // image column of pt column 0
    const int We = W + D - 1, sc0 = x0 - d0 + D - DC;
    constexpr int NPR = (SH * PRW + kCostThreads - 1) / kCostThreads;
    constexpr int NPT = (SH * PTW + kCostThreads - 1) / kCostThreads;
    constexpr int NSB = (kCostTY * kCostSW + kCostThreads - 1) / kCostThreads;
    {
        float2 vr[NPR], vt[NPT], vs[NSB];
#pragma unroll
        for (int it = 0; it < NPR; ++it) {
            const int i = threadIdx.x + it * kCostThreads, r = i / PRW, c = i - r * PRW;
            const float *row = R + (size_t)clampi(y0 - rw + r, 0, H - 1) * W;
            const int x = x0 - rw + c;
            if (i < SH * PRW) vr[it] = make_float2(row[clampi(x, 0, W - 1)], row[clampi(x + 32, 0, W - 1)]);
        }
#pragma unroll
        for (int it = 0; it < NPT; ++it) {
            const int i = threadIdx.x + it * kCostThreads, r = i / PTW, c = i - r * PTW;
            const float *row = T + (size_t)clampi(y0 - rw + r, 0, H - 1) * W;
            if (i < SH * PTW) vt[it] = make_float2(row[clampi(tc0 + c, 0, W - 1)], row[clampi(tc0 + c + 32, 0, W - 1)]);
        }
        // the target statistics the tile's epilogue reads: row v, columns u - d + D - 1 of the
        // extended grid, entry (u - x0) - (d - d0) + DC - 1
#pragma unroll
        for (int it = 0; it < NSB; ++it) {
            const int i = threadIdx.x + it * kCostThreads, r = i / kCostSW, c = i - r * kCostSW;
            const int v = y0 + r, xe = sc0 + c;
            const bool ok = i < kCostTY * kCostSW && v < H && xe >= 0 && xe < We;
            const size_t so = ((size_t)b * H + (ok ? v : 0)) * We + (ok ? xe : 0);
            vs[it] = ok ? make_float2(mut[so], isdt[so]) : make_float2(0.f, 0.f);   // (mu_b, 1 / s_b)
        }
#pragma unroll
        for (int it = 0; it < NPR; ++it) {
            const int i = threadIdx.x + it * kCostThreads;
            if (i < SH * PRW) pr[i] = vr[it];
        }
#pragma unroll
        for (int it = 0; it < NPT; ++it) {
            const int i = threadIdx.x + it * kCostThreads;
            if (i < SH * PTW) pt[i] = vt[it];
        }
#pragma unroll
        for (int it = 0; it < NSB; ++it) {
            const int i = threadIdx.x + it * kCostThreads;
            if (i < kCostTY * kCostSW) {
                smb[i] = vs[it].x;
                ssb[i] = vs[it].y;
            }
        }
    }
    __syncthreads();
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const int u0 = x0 + tx, v0 = y0 + 2 * ty;
    auto inside = [&](int h, int j) { return u0 + 32 * j < W && v0 + h < H; };
    float2 ma[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        float m2[2] = {0.f, 0.f};
#pragma unroll
        for (int j = 0; j < 2; ++j)
            if (inside(h, j)) m2[j] = mur[b * HW + (size_t)(v0 + h) * W + u0 + 32 * j];
        ma[h] = make_float2(m2[0], m2[1]);
    }
    float2 acc[2][DC], asum[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        asum[h] = make_float2(0.f, 0.f);
#pragma unroll
        for (int k = 0; k < DC; ++k) acc[h][k] = make_float2(0.f, 0.f);
    }
    // image row y of the thread's halo (tile row 2 ty + y): window row y of pixel row 0 and
    // window row y - 1 of pixel row 1
    auto row = [&](int y, auto h0_c, auto h1_c) {
        constexpr bool H0 = decltype(h0_c)::value, H1 = decltype(h1_c)::value;
        const float2 *rrow = pr + (2 * ty + y) * PRW + tx;
        const float2 *trow = pt + (2 * ty + y) * PTW + tx + (DC - 1);
        float2 win[DC];                      // win[k] = trow[dx - k]
#pragma unroll
        for (int k = 0; k < DC; ++k) win[k] = trow[-k];
#pragma unroll
        for (int dx = 0; dx < w; ++dx) {
            if (dx > 0) {
#pragma unroll
                for (int k = DC - 1; k > 0; --k) win[k] = win[k - 1];
                win[0] = trow[dx];
            }
            const float2 r = rrow[dx];
            if constexpr (H0) {
                const float2 a = __fadd2_rn(r, make_float2(-ma[0].x, -ma[0].y));
                asum[0] = __fadd2_rn(asum[0], a);
#pragma unroll
                for (int k = 0; k < DC; ++k) acc[0][k] = __ffma2_rn(a, win[k], acc[0][k]);
            }
            if constexpr (H1) {
                const float2 a = __fadd2_rn(r, make_float2(-ma[1].x, -ma[1].y));
                asum[1] = __fadd2_rn(asum[1], a);
#pragma unroll
                for (int k = 0; k < DC; ++k) acc[1][k] = __ffma2_rn(a, win[k], acc[1][k]);
            }
        }
    };
    row(0, std::true_type(), std::false_type());
#pragma unroll 1
    for (int y = 1; y < w; ++y) row(y, std::true_type(), std::true_type());
    row(w, std::false_type(), std::true_type());

    const float n = (float)(w * w);
#pragma unroll
    for (int h = 0; h < 2; ++h)
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            if (!inside(h, j)) continue;
            const int u = u0 + 32 * j, v = v0 + h;
            const float sav = sdr[b * HW + (size_t)v * W + u], as = j ? asum[h].y : asum[h].x;
            const float ia = sav > 0.f ? 1.f / (n * sav) : 0.f;   // 1 / (n s_a), once per pixel
#pragma unroll
            for (int k = 0; k < DC; ++k) {
                const int d = d0 + k;
                if (d >= D) break;
                const int e = (2 * ty + h) * kCostSW + tx + 32 * j - k + DC - 1;
                const float mb = smb[e], isb = ssb[e];
                const float ak = j ? acc[h][k].y : acc[h][k].x;
                float c = 1.f;
                if (ia > 0.f && isb > 0.f) c = 1.f - fmaf(-mb, as, ak) * ia * isb;
                cost[((size_t)b * D + d) * HW + (size_t)v * W + u] = c;
            }
        }
}

// ------------------------------------------------------------------ aggregation stencil
struct AggArgs {
    const float *img;      // reference image [B][H][W]
    const float *vol;      // neighbour values [B][D][H][W]: the cost (FWD, H) or h (GC)
    const float *shift;    // FWD: row shifts
    float *disp;           // FWD: l
    float *lse, *lbar;     // FWD out, H in
    const float *gdisp;    // H: dS/dl
    float *h;              // H out
    float *beta, *t1;      // H out, GC in
    float *gc;             // GC out
    const float *cost;     // GC: c(x, d) of the centre pixel
    float *gw;             // GC out: image gradient through the weights
    int W, H, D;
    int warp_mode;         // FWD: the add-back is s_i (rounded) or s(v) (linear warp)
    float kappa;           // sqrt(log2 e) / sigma1: scaled intensities
    float k0;              // -log2 e / sigma0^2
    float kT;              // log2 e / T
    float invT;            // 1 / T
    float gw_scale;        // 2 / (sigma1^2 kappa)
};

// The disparity chunks of a tile are staged in two shared-memory buffers: while chunk k is
// aggregated, the copies of chunk k + 1 are in flight (cp.async, 4 bytes per element, zero
// fill outside the image and beyond D).
__device__ __forceinline__ void cp_async4(void *dst, const void *src, bool valid)
{
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(d), "l"(src), "r"(valid ? 4 : 0)
                 : "memory");
}

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }

template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// One tile per block (agg_tx x agg_ty); thread (tx, ty) owns the pixels (x0 + tx, y0 + R ty + i),
// i < R = agg_rows(MODE), and kAggDC disparities at a time.  The weights of eq. (omega_s) are formed as
// exp2(kx + ky - (sI_p - sI_q)^2) with sI = kappa I; an out-of-image neighbour has
// sI = kFar and a zero value, so its weight and every product with it are exactly 0.
template <int MODE, int RB>
__global__ void __launch_bounds__(agg_threads(MODE), MODE == AGG_FWD ? 3 : MODE == AGG_GC ? 2 : 1) k_dagg(const AggArgs a)
{
    constexpr int ROWS = agg_rows(MODE);
    constexpr int DC = kAggDC, NQ = DC / 4, NR = ROWS + 2 * RB;
    constexpr bool DB = agg_dbuf(MODE);
    constexpr int kAggTX = agg_tx(MODE), kAggTY = agg_ty(MODE), kAggThreads = agg_threads(MODE);
    constexpr int TW = kAggTX + 2 * RB, TH = kAggTY + 2 * RB;
    constexpr bool TWO = MODE != AGG_FWD;
    extern __shared__ float4 smem4[];
    float4 *Vbuf = smem4;                                     // [1 or 2][NQ][TH][TW]
    float *sI = (float *)(Vbuf + (DB ? 2 : 1) * NQ * TH * TW); // [TH][TW]
    float *scst = sI + TH * TW;                                  // AGG_GC: [DC][agg_ty][agg_tx], c(x, d)
    const int b = blockIdx.z, x0 = blockIdx.x * kAggTX, y0 = blockIdx.y * kAggTY;
    constexpr int WCOL = kAggTX / 32;               // warp columns of the tile
    const int warp = threadIdx.x >> 5;
    const int tx = (warp % WCOL) * 32 + (threadIdx.x & 31), ty = warp / WCOL;
    const int W = a.W, H = a.H, D = a.D;
    const size_t HW = (size_t)H * W;
    const float *img = a.img + b * HW;
    auto issue_chunk = [&](int d0, float4 *V) {
        for (int i = threadIdx.x; i < TH * TW; i += kAggThreads) {
            const int r = i / TW, c = i - r * TW, y = y0 - RB + r, x = x0 - RB + c;
            const bool in = y >= 0 && y < H && x >= 0 && x < W;
            const float *src = a.vol + ((size_t)b * D) * HW + (in ? (size_t)y * W + x : 0);
#pragma unroll
            for (int q = 0; q < NQ; ++q) {
                float *dst = reinterpret_cast<float *>(&V[(q * TH + r) * TW + c]);
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int d = d0 + 4 * q + j;
                    const bool ok = in && d < D;
                    cp_async4(dst + j, ok ? src + (size_t)d * HW : a.vol, ok);
                }
            }
        }
        if constexpr (MODE == AGG_GC) {
            // the centre pixels' costs of the chunk, read by the chunk's epilogue
            for (int i = threadIdx.x; i < DC * kAggTY * kAggTX; i += kAggThreads) {
                const int k = i / (kAggTY * kAggTX), rc = i - k * (kAggTY * kAggTX);
                const int r = rc / kAggTX, c = rc - r * kAggTX, y = y0 + r, x = x0 + c, d = d0 + k;
                const bool ok = y < H && x < W && d < D;
                cp_async4(scst + i, ok ? a.cost + ((size_t)b * D + d) * HW + (size_t)y * W + x : a.cost, ok);
            }
        }
        cp_async_commit();
    };
    if constexpr (DB) issue_chunk(0, Vbuf);
    {
        // every load of a thread before its first store: the loads are in flight together
        constexpr int NI = (TH * TW + kAggThreads - 1) / kAggThreads;
        float vi[NI];
#pragma unroll
        for (int it = 0; it < NI; ++it) {
            const int i = threadIdx.x + it * kAggThreads, r = i / TW, c = i - r * TW;
            const int y = y0 - RB + r, x = x0 - RB + c;
            vi[it] = (i < TH * TW && y >= 0 && y < H && x >= 0 && x < W) ? img[(size_t)y * W + x] * a.kappa : kFar;
        }
#pragma unroll
        for (int it = 0; it < NI; ++it) {
            const int i = threadIdx.x + it * kAggThreads;
            if (i < TH * TW) sI[i] = vi[it];
        }
    }
    float ky[2 * RB + 1];
#pragma unroll
    for (int j = 0; j <= 2 * RB; ++j) ky[j] = a.k0 * (float)((j - RB) * (j - RB));
    __syncthreads();

    const int px = x0 + tx;
    float sIp[ROWS];
    int py[ROWS];
    bool pin[ROWS];
#pragma unroll
    for (int i = 0; i < ROWS; ++i) {
        py[i] = y0 + ROWS * ty + i;
        pin[i] = px < W && py[i] < H;
        sIp[i] = sI[(ROWS * ty + i + RB) * TW + tx + RB];
    }
    // per-pixel state across chunks
    float st0[ROWS], st1[ROWS], st2[ROWS], st3[ROWS];
#pragma unroll
    for (int i = 0; i < ROWS; ++i) {
        st0[i] = st1[i] = st2[i] = st3[i] = 0.f;
        if constexpr (MODE == AGG_FWD) st0[i] = -INFINITY;   // running max of -E kT
        if (MODE == AGG_H && pin[i]) {
            const size_t o = b * HW + (size_t)py[i] * W + px;
            st0[i] = a.gdisp[o];                             // gl
            st1[i] = a.lse[o];                               // log2-sum-exp
            st2[i] = a.lbar[o];                              // soft-argmin without the shift
        }
    }
    float S[ROWS];          // sum_q w (sI_q - sI_p), the same in every chunk
    float Z[ROWS];          // sum_q w, the same in every chunk
    float invZ[ROWS];
    // Z and S depend on no disparity: the first chunk sums them (the same terms in the same
    // order as any chunk would) and later chunks reuse them
    float beta[ROWS], tacc[ROWS];
#pragma unroll
    for (int i = 0; i < ROWS; ++i) S[i] = beta[i] = tacc[i] = 0.f;

    for (int d0 = 0, kc = 0; d0 < D; d0 += DC, ++kc) {
        const float4 *V = Vbuf + (DB ? (kc & 1) * NQ * TH * TW : 0);
        if constexpr (DB) {
            if (d0 + DC < D) {
                issue_chunk(d0 + DC, Vbuf + ((kc + 1) & 1) * NQ * TH * TW);
                cp_async_wait<1>();      // this chunk's copies are complete
            } else {
                cp_async_wait<0>();
            }
        } else {
            issue_chunk(d0, Vbuf);
            cp_async_wait<0>();
        }
        __syncthreads();

        // accumulators in pairs of disparities (packed f32x2 FMAs)
        float2 acc0[ROWS][DC / 2], acc1[ROWS][TWO ? DC / 2 : 1];
#pragma unroll
        for (int i = 0; i < ROWS; ++i) {
            if (kc == 0) {
                Z[i] = 0.f;
                if constexpr (TWO) S[i] = 0.f;
            }
#pragma unroll
            for (int k = 0; k < DC / 2; ++k) {
                acc0[i][k] = make_float2(0.f, 0.f);
                if constexpr (TWO) acc1[i][k] = make_float2(0.f, 0.f);
            }
        }
        auto accumulate = [&](auto first_c) {
            constexpr bool FIRST = decltype(first_c)::value;
#pragma unroll 1
            for (int dx = -RB; dx <= RB; ++dx) {
                const float kx = a.k0 * (float)(dx * dx);
                const int col = tx + RB + dx;
#pragma unroll
                for (int r = 0; r < NR; ++r) {
                    const int srow = ROWS * ty + r;
                    const float sq = sI[srow * TW + col];
                    float4 v4[NQ];
#pragma unroll
                    for (int q = 0; q < NQ; ++q) v4[q] = V[(q * TH + srow) * TW + col];
#pragma unroll
                    for (int i = 0; i < ROWS; ++i) {
                        const int dy = r - RB - i;
                        if (dy < -RB || dy > RB) continue;
                        const float dd = sIp[i] - sq;
                        const float w = ex2_fast(fmaf(-dd, dd, kx + ky[dy + RB]));
                        if constexpr (FIRST) Z[i] += w;
                        const float2 w2 = make_float2(w, w);
#pragma unroll
                        for (int q = 0; q < NQ; ++q) {
                            acc0[i][2 * q + 0] = __ffma2_rn(w2, make_float2(v4[q].x, v4[q].y), acc0[i][2 * q + 0]);
                            acc0[i][2 * q + 1] = __ffma2_rn(w2, make_float2(v4[q].z, v4[q].w), acc0[i][2 * q + 1]);
                        }
                        if constexpr (TWO) {
                            const float wd = -w * dd;
                            if constexpr (FIRST) S[i] += wd;
                            const float2 wd2 = make_float2(wd, wd);
#pragma unroll
                            for (int q = 0; q < NQ; ++q) {
                                acc1[i][2 * q + 0] = __ffma2_rn(wd2, make_float2(v4[q].x, v4[q].y), acc1[i][2 * q + 0]);
                                acc1[i][2 * q + 1] = __ffma2_rn(wd2, make_float2(v4[q].z, v4[q].w), acc1[i][2 * q + 1]);
                            }
                        }
                    }
                }
            }
        };
        if constexpr (MODE == AGG_GC) {
            accumulate(std::false_type());   // (Z and S serve the other two modes only)
        } else if (kc == 0) {
            accumulate(std::true_type());
#pragma unroll
            for (int i = 0; i < ROWS; ++i) invZ[i] = 1.f / Z[i];
        } else {
            accumulate(std::false_type());
        }

        // chunk epilogue
#pragma unroll
        for (int i = 0; i < ROWS; ++i) {
            if (!pin[i]) continue;
            const size_t pix = (size_t)py[i] * W + px;
            if constexpr (MODE == AGG_FWD) {
                float z[DC], mc = st0[i];
#pragma unroll
                for (int k = 0; k < DC; ++k) {
                    z[k] = -(lane(acc0[i][k >> 1], k) * invZ[i]) * a.kT;
                    if (d0 + k < D) mc = fmaxf(mc, z[k]);
                }
                const float sc = exp2f(st0[i] - mc);
                float s0 = st1[i] * sc, s1 = st2[i] * sc;
#pragma unroll
                for (int k = 0; k < DC; ++k) {
                    if (d0 + k >= D) break;
                    const float e = exp2f(z[k] - mc);
                    s0 += e;
                    s1 = fmaf((float)(d0 + k), e, s1);
                }
                st0[i] = mc;
                st1[i] = s0;
                st2[i] = s1;
            } else if constexpr (MODE == AGG_H) {
#pragma unroll
                for (int k = 0; k < DC; ++k) {
                    const int d = d0 + k;
                    if (d >= D) break;
                    const float E = lane(acc0[i][k >> 1], k) * invZ[i];
                    const float P = exp2f(-E * a.kT - st1[i]);
                    const float hv = -st0[i] * a.invT * P * ((float)d - st2[i]) * invZ[i];
                    a.h[((size_t)b * D + d) * HW + pix] = hv;
                    beta[i] = fmaf(hv, E, beta[i]);
                    tacc[i] = fmaf(hv, lane(acc1[i][k >> 1], k), tacc[i]);
                }
            } else {
#pragma unroll
                for (int k = 0; k < DC; ++k) {
                    const int d = d0 + k;
                    if (d >= D) break;
                    const size_t o = ((size_t)b * D + d) * HW + pix;
                    a.gc[o] = lane(acc0[i][k >> 1], k);
                    const float cx = scst[(k * kAggTY + ROWS * ty + i) * kAggTX + tx];
                    tacc[i] = fmaf(cx, lane(acc1[i][k >> 1], k), tacc[i]);
                }
            }
        }
        __syncthreads();   // every thread is done with this buffer before it is refilled
    }

    if constexpr (MODE == AGG_FWD) {
#pragma unroll
        for (int i = 0; i < ROWS; ++i) {
            if (!pin[i]) continue;
            const size_t o = b * HW + (size_t)py[i] * W + px;
            const float lbar = st2[i] / st1[i];
            a.lbar[o] = lbar;
            a.lse[o] = st0[i] + log2f(st1[i]);
            const float sv = a.shift[(size_t)b * H + py[i]];
            a.disp[o] = lbar + (a.warp_mode == STEREO_WARP_LINEAR ? sv : row_shift_value(sv));
        }
        return;
    }
    if constexpr (MODE == AGG_H) {
#pragma unroll
        for (int i = 0; i < ROWS; ++i) {
            if (!pin[i]) continue;
            const size_t o = b * HW + (size_t)py[i] * W + px;
            a.beta[o] = beta[i];
            a.t1[o] = fmaf(-beta[i], S[i], tacc[i]);
        }
        return;
    }
    // AGG_GC: the weights' term of beta, sum_q w (sI_q - sI_x) beta(q), over a staged tile
    __syncthreads();
    float *sb = (float *)Vbuf;
    for (int i = threadIdx.x; i < TH * TW; i += kAggThreads) {
        const int r = i / TW, c = i - r * TW, y = y0 - RB + r, x = x0 - RB + c;
        const bool in = y >= 0 && y < H && x >= 0 && x < W;
        cp_async4(sb + i, in ? a.beta + b * HW + (size_t)y * W + x : a.beta, in);
    }
    cp_async_commit();
    cp_async_wait<0>();
    __syncthreads();
    float sbeta[ROWS];
#pragma unroll
    for (int i = 0; i < ROWS; ++i) sbeta[i] = 0.f;
#pragma unroll 1
    for (int dx = -RB; dx <= RB; ++dx) {
        const float kx = a.k0 * (float)(dx * dx);
        const int col = tx + RB + dx;
#pragma unroll
        for (int r = 0; r < NR; ++r) {
            const int srow = ROWS * ty + r;
            const float sq = sI[srow * TW + col], bq = sb[srow * TW + col];
#pragma unroll
            for (int i = 0; i < ROWS; ++i) {
                const int dy = r - RB - i;
                if (dy < -RB || dy > RB) continue;
                const float dd = sIp[i] - sq;
                const float w = ex2_fast(fmaf(-dd, dd, kx + ky[dy + RB]));
                sbeta[i] = fmaf(-w * dd, bq, sbeta[i]);
            }
        }
    }
    float t1v[ROWS];   // (all loads before the first store)
#pragma unroll
    for (int i = 0; i < ROWS; ++i) t1v[i] = pin[i] ? a.t1[b * HW + (size_t)py[i] * W + px] : 0.f;
#pragma unroll
    for (int i = 0; i < ROWS; ++i) {
        if (!pin[i]) continue;
        const size_t o = b * HW + (size_t)py[i] * W + px;
        a.gw[o] = a.gw_scale * (t1v[i] + tacc[i] - sbeta[i]);
    }
}

// ------------------------------------------------------------------ cost adjoint
struct CbArgs {
    const float *ref, *tw, *mur, *sdr, *mut, *isdt, *cost, *gc;
    float *gpart;          // [B][Hr][tile column][32 + D - 1] partial diagonal sums of Gamma (or null)
    float *grefx;
    int W, H, D, Wr, Hr, We;
    float inv_n;
};

// Extended reference positions X in [-rw, W-1+rw] x [-rw, H-1+rw], a 32 x kCbTY tile per block
// (a thread owns two of its rows, 8 apart).
// kCbDC disparities at a time: the four window-pair terms A, A mu_a, C, C mu_b of the pairs q
// in the tile's halo are staged and box-summed with running sums (along rows, then along
// columns); the d-independent terms of the reference gradient are summed over d per q and
// box-summed once at the end.  Row strides are padded to odd lengths so that the running
// sums of neighbouring rows hit distinct shared-memory banks.  Gamma(X, d) is added into a
// shared row per tile row at entry X - X0 - d + D - 1 (within one step of d every lane of a
// warp meets a distinct entry; the two steps of a round are ordered by a warp barrier, the
// rounds by the block's), and the tile's rows of partial sums are written once at the end.
constexpr int kCbDC = 2;
constexpr int kCbTY = 16;   // extended rows per tile (two per thread, 8 apart)

// Running box sums of one half of a plane row: out[x] = sum_{j < WN} in[x + j], x < 16.
template <int WN>
__device__ __forceinline__ void row_box16(const float *in, float *out)
{
    float s = 0.f;
#pragma unroll
    for (int j = 0; j < WN; ++j) s += in[j];
    out[0] = s;
#pragma unroll
    for (int x = 1; x < 16; ++x) {
        s += in[x + WN - 1] - in[x - 1];
        out[x] = s;
    }
}

// Running box sums of one plane row: out[x] = sum_{j < WN} in[x + j], x < 32.
template <int WN>
__device__ __forceinline__ void row_box(const float *in, float *out)
{
    float s = 0.f;
#pragma unroll
    for (int j = 0; j < WN; ++j) s += in[j];
    out[0] = s;
#pragma unroll 8
    for (int x = 1; x < 32; ++x) {
        s += in[x + WN - 1] - in[x - 1];
        out[x] = s;
    }
}

template <int RW>
__global__ void __launch_bounds__(256, 2) k_dcost_bwd(const CbArgs a)
{
    constexpr int TY = kCbTY, RPT = TY / 8;                     // tile rows; rows per thread (8 apart)
    constexpr int QW = 32 + 2 * RW, QH = TY + 2 * RW, NQ = QW * QH, NS = (NQ + 255) / 256;
    constexpr int WN = 2 * RW + 1, DC = kCbDC, NP = 4 * DC;   // planes: 4 terms x DC disparities
    constexpr int SW = QW | 1, SP = SW * QH;                    // staged row stride (odd), plane size
    constexpr int HW_ = 33, HP = HW_ * QH;                      // row-summed row stride (odd), plane size
    extern __shared__ float cb_smem[];
    float *st = cb_smem;                       // [NP][QH][SW]
    float *hb = st + NP * SP;                  // [NP][QH][33]
    float *vb = hb + NP * HP;                  // [NP][TY][32]
    float *gts = vb + NP * TY * 32;            // [TY][32 + D - 1] partial diagonal sums
    const int b = blockIdx.z;
    const int W = a.W, H = a.H, D = a.D;
    const size_t HW = (size_t)H * W;
    const int X0 = blockIdx.x * 32 - RW, Y0 = blockIdx.y * TY - RW;   // image coords of the tile origin
    float qmu[NS], qisa[NS], sAmb[NS], sB[NS], sBmu[NS];
    size_t vbase[NS], sbase[NS];       // cost / gc entry of (q, d = 0); statistics entry of (q, 0)
    int qofs[NS];                      // q's offset inside a staged plane
    bool qin[NS];
    // The halo's pairs q are taken in 32-column slabs (a warp's lanes on one staged row of the
    // first slab), then the 2 RW columns to its right.
#pragma unroll
    for (int s = 0; s < NS; ++s) {
        const int j = threadIdx.x + 256 * s;
        int r, c;
        if (j < QH * 32) {
            r = j >> 5;
            c = j & 31;
        } else {
            const int j2 = j - QH * 32;
            r = RW > 0 ? j2 / (2 * RW) : 0;
            c = RW > 0 ? 32 + j2 % (2 * RW) : 0;
        }
        const int qy = Y0 - RW + r, qx = X0 - RW + c;
        qin[s] = j < NQ && qy >= 0 && qy < H && qx >= 0 && qx < W;
        qofs[s] = j < NQ ? r * SW + c : 0;
        const size_t qo = qin[s] ? (size_t)qy * W + qx : 0;
        vbase[s] = (size_t)b * D * HW + qo;
        sbase[s] = qin[s] ? ((size_t)b * H + qy) * a.We + qx + D - 1 : 0;
        qmu[s] = qin[s] ? a.mur[b * HW + qo] : 0.f;
        const float sa = qin[s] ? a.sdr[b * HW + qo] : 0.f;
        qisa[s] = sa > 0.f ? __frcp_rn(sa) : 0.f;       // 0 marks a flat reference block
        sAmb[s] = sB[s] = sBmu[s] = 0.f;
    }
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const int X = X0 + tx;
    float rv[RPT], gacc[RPT];
    bool xin[RPT];
    const float *twrow[RPT];
#pragma unroll
    for (int i = 0; i < RPT; ++i) {
        const int Y = Y0 + ty + 8 * i;
        xin[i] = X <= W - 1 + RW && Y <= H - 1 + RW;
        const int yc = clampi(Y, 0, H - 1);
        rv[i] = a.ref[b * HW + (size_t)yc * W + clampi(X, 0, W - 1)];
        twrow[i] = a.tw + b * HW + (size_t)yc * W;
        gacc[i] = 0.f;
    }
    const int GW = cb_diag_w(D);
    if (a.gpart)
        for (int i = threadIdx.x; i < TY * GW; i += 256) gts[i] = 0.f;   // (the first round's barriers order these)
    // the loads of a round are issued one round ahead, so that they are in flight while the
    // previous round's box sums run
    float g[NS][DC], cc[NS][DC], sb[NS][DC], mb[NS][DC];
    // the target values t(X - d) of the tile rows, loaded a round ahead too (but for the widest
    // window, whose registers they would spill)
    constexpr bool TPF = RW < 7;
    float tn[RPT][DC];
    auto load_round = [&](int d0) {
        if constexpr (TPF) {
#pragma unroll
            for (int i = 0; i < RPT; ++i)
#pragma unroll
                for (int k = 0; k < DC; ++k)
                    tn[i][k] = (xin[i] && d0 + k < D) ? twrow[i][clampi(X - d0 - k, 0, W - 1)] : 0.f;
        }
#pragma unroll
        for (int s = 0; s < NS; ++s)
#pragma unroll
            for (int k = 0; k < DC; ++k) {
                const bool ok = qin[s] && d0 + k < D;
                const size_t vo = vbase[s] + (size_t)(ok ? d0 + k : 0) * HW, so = sbase[s] - (ok ? d0 + k : 0);
                g[s][k] = ok ? a.gc[vo] : 0.f;
                cc[s][k] = ok ? a.cost[vo] : 1.f;
                sb[s][k] = ok ? a.isdt[so] : 0.f;   // 1 / s_b (0: a flat target block)
                mb[s][k] = ok ? a.mut[so] : 0.f;
            }
    };
    load_round(0);
    for (int d0 = 0; d0 < D; d0 += DC) {
        // ---- stage the window-pair terms of the halo for DC disparities
#pragma unroll
        for (int s = 0; s < NS; ++s) {
            const int j = threadIdx.x + 256 * s;
            if (j >= NQ) break;
#pragma unroll
            for (int k = 0; k < DC; ++k) {
                float A = 0.f, C = 0.f, Bq = 0.f;
                if (qisa[s] > 0.f && sb[s][k] > 0.f) {
                    const float isb = sb[s][k];
                    const float gn = g[s][k] * a.inv_n, gnc = gn * (1.f - cc[s][k]);
                    A = -gn * qisa[s] * isb;
                    Bq = gnc * qisa[s] * qisa[s];
                    C = gnc * isb * isb;
                }
                sAmb[s] = fmaf(A, mb[s][k], sAmb[s]);
                sB[s] += Bq;
                sBmu[s] = fmaf(Bq, qmu[s], sBmu[s]);
                st[(0 * DC + k) * SP + qofs[s]] = A;
                st[(1 * DC + k) * SP + qofs[s]] = A * qmu[s];
                st[(2 * DC + k) * SP + qofs[s]] = C;
                st[(3 * DC + k) * SP + qofs[s]] = C * mb[s][k];
            }
        }
        float tc[RPT][DC];
        if constexpr (TPF) {
#pragma unroll
            for (int i = 0; i < RPT; ++i)
#pragma unroll
                for (int k = 0; k < DC; ++k) tc[i][k] = tn[i][k];
        }
        if (d0 + DC < D) load_round(d0 + DC);
        __syncthreads();
        // ---- box sums along rows: one running sum per (plane, halo row, half row); with the
        // odd row strides the 32 lanes of a warp (16 rows, both halves) meet 32 distinct banks
        for (int t = threadIdx.x; t < NP * QH * 2; t += 256) {
            const int half = t & 1, pr = t >> 1;
            const int p = pr / QH, row = pr - p * QH;
            row_box16<WN>(st + p * SP + row * SW + 16 * half, hb + p * HP + row * HW_ + 16 * half);
        }
        __syncthreads();
        // ---- box sums along columns: one running sum per (plane, column) over the TY tile rows
        for (int t = threadIdx.x; t < NP * 32; t += 256) {
            const int p = t >> 5, xc = t & 31;
            const float *col = hb + p * HP + xc;
            float *out = vb + p * TY * 32 + xc;
            float s = 0.f;
#pragma unroll
            for (int i = 0; i < WN; ++i) s += col[i * HW_];
            out[0] = s;
#pragma unroll
            for (int y = 1; y < TY; ++y) {
                s += col[(y + WN - 1) * HW_] - col[(y - 1) * HW_];
                out[y * 32] = s;
            }
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < DC; ++k) {
            const int d = d0 + k;
#pragma unroll
            for (int i = 0; i < RPT; ++i) {
                const int o = (ty + 8 * i) * 32 + tx;
                const float bA = vb[(0 * DC + k) * TY * 32 + o], bAm = vb[(1 * DC + k) * TY * 32 + o];
                const float bC = vb[(2 * DC + k) * TY * 32 + o], bCm = vb[(3 * DC + k) * TY * 32 + o];
                if (xin[i] && d < D) {
                    const float t = TPF ? tc[i][k] : twrow[i][clampi(X - d, 0, W - 1)];
                    if (a.gpart) gts[(ty + 8 * i) * GW + tx - d + D - 1] += fmaf(rv[i], bA, -bAm) + fmaf(t, bC, -bCm);
                    gacc[i] = fmaf(t, bA, gacc[i]);
                }
            }
            __syncwarp();   // lane x at d + 1 meets the entry of lane x - 1 at d
        }
        // the next round's staging writes st only: hb and vb are rewritten after its barrier
    }
    // the d-independent terms: - box(sum_d A mu_b) + r box(sum_d B) - box(sum_d B mu_a)
    __syncthreads();
    if (a.gpart) {
        // this tile's partial diagonal sums, one row per tile row inside the extended grid
        const int nbx = cb_tiles_x(a.Wr);
        for (int i = threadIdx.x; i < TY * GW; i += 256) {
            const int r = i / GW, j = i - r * GW, row = blockIdx.y * TY + r;
            if (row < a.Hr) a.gpart[(((size_t)b * a.Hr + row) * nbx + blockIdx.x) * GW + j] = gts[i];
        }
    }
#pragma unroll
    for (int s = 0; s < NS; ++s) {
        const int j = threadIdx.x + 256 * s;
        if (j >= NQ) break;
        st[0 * SP + qofs[s]] = sAmb[s];
        st[1 * SP + qofs[s]] = sB[s];
        st[2 * SP + qofs[s]] = sBmu[s];
    }
    __syncthreads();
    for (int t = threadIdx.x; t < 3 * QH; t += 256) {
        const int p = t / QH, row = t - p * QH;
        row_box<WN>(st + p * SP + row * SW, hb + p * HP + row * HW_);
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < RPT; ++i) {
        float bx[3];
#pragma unroll
        for (int qn = 0; qn < 3; ++qn) {
            const float *col = hb + qn * HP + (ty + 8 * i) * HW_ + tx;
            float sum = 0.f;
#pragma unroll
            for (int j = 0; j < WN; ++j) sum += col[j * HW_];
            bx[qn] = sum;
        }
        const int Y = Y0 + ty + 8 * i;
        if (xin[i])
            a.grefx[((size_t)b * a.Hr + (Y + RW)) * a.Wr + (X + RW)] = gacc[i] - bx[0] + fmaf(rv[i], bx[1], -bx[2]);
    }
}


// Target positions Xt in [-rw-(D-1), W-1+rw] (column c = Xt + rw + D - 1): the sum over d of
// Gamma(Xt + d, d), as the partial sums of the cost adjoint's tiles whose columns reach it
// (tile bx holds c in entry c - 32 bx), added in tile order.
__global__ void __launch_bounds__(256) k_dtgt_diag(const float *__restrict__ gpart, float *__restrict__ gtwx,
                                                   int D, int Wr, int Hr, int Wt)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x, row = blockIdx.y, b = blockIdx.z;
    if (c >= Wt) return;
    const int GW = cb_diag_w(D), nbx = cb_tiles_x(Wr);
    const int bxlo = max(0, (c - GW + 1 + 31) / 32), bxhi = min(nbx - 1, c / 32);
    const float *p = gpart + ((size_t)b * Hr + row) * nbx * GW;
    float s = 0.f;
    for (int bx = bxlo; bx <= bxhi; ++bx) s += p[(size_t)bx * GW + c - 32 * bx];
    gtwx[((size_t)b * Hr + row) * Wt + c] = s;
}

// The folded gradient of the warped target at column xw of row y: every extended target
// position Xt that reads column xw after clamping (the whole left or right overhang at the
// edges), over the rows that clamp to y.
__device__ __forceinline__ float fold_tw(const float *__restrict__ gtwx, int b, int xw, int ylo, int yhi, int W,
                                         int D, int rw, int Hr, int Wt)
{
    const int tlo = xw == 0 ? -rw - (D - 1) : xw, thi = xw == W - 1 ? W - 1 + rw : xw;
    float s = 0.f;
    for (int Y = ylo; Y <= yhi; ++Y) {
        const float *row = gtwx + ((size_t)b * Hr + Y + rw) * Wt + rw + (D - 1);
        for (int Xt = tlo; Xt <= thi; ++Xt) s += row[Xt];
    }
    return s;
}

// The sum, over the warped columns xw that read source column x through clamp(xw - si),
// of the folded warped-target gradient: the adjoint of one integer-shift gather.
__device__ __forceinline__ float unwarp_sum(const float *__restrict__ gtwx, int b, int x, int si, int ylo, int yhi,
                                            int W, int D, int rw, int Hr, int Wt)
{
    int lo, hi;
    if (W == 1) {
        lo = 0;
        hi = 0;
    } else if (x == 0) {
        lo = 0;
        hi = min(W - 1, si);
    } else if (x == W - 1) {
        lo = max(0, W - 1 + si);
        hi = W - 1;
    } else {
        lo = hi = x + si;
        if (lo < 0 || lo > W - 1) {
            lo = 1;
            hi = 0;
        }
    }
    float s = 0.f;
    for (int xw = lo; xw <= hi; ++xw) s += fold_tw(gtwx, b, xw, ylo, yhi, W, D, rw, Hr, Wt);
    return s;
}

// Fold the extended grids back onto the image (every clamp-to-edge position adds to the
// edge pixel it read) and undo the warp (every warped column adds to the column it read;
// the linear warp reads two columns, with weights 1 - f and f).
__global__ void __launch_bounds__(256) k_dfold(const float *__restrict__ grefx, const float *__restrict__ gw,
                                               const float *__restrict__ gtwx, const float *__restrict__ shift,
                                               float *__restrict__ gref, float *__restrict__ gtgt, int W, int H,
                                               int D, int rw, int Wr, int Hr, int Wt, int mode)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y, b = blockIdx.z;
    if (x >= W) return;
    const size_t pix = ((size_t)b * H + y) * W + x;
    const int ylo = y == 0 ? -rw : y, yhi = y == H - 1 ? H - 1 + rw : y;
    if (gref) {
        const int xlo = x == 0 ? -rw : x, xhi = x == W - 1 ? W - 1 + rw : x;
        float s = 0.f;
        for (int Y = ylo; Y <= yhi; ++Y)
            for (int X = xlo; X <= xhi; ++X) s += grefx[((size_t)b * Hr + Y + rw) * Wr + X + rw];
        gref[pix] = s + gw[pix];
    }
    if (gtgt) {
        const float sv = shift[(size_t)b * H + y];
        if (mode == STEREO_WARP_LINEAR) {
            // tw(xw) = (1 - f) tgt(clamp(xw + k)) + f tgt(clamp(xw + k + 1))
            const LinShift ls = lin_shift(sv, W);
            const float ga = unwarp_sum(gtwx, b, x, -ls.k, ylo, yhi, W, D, rw, Hr, Wt);
            const float gb = unwarp_sum(gtwx, b, x, -ls.k - 1, ylo, yhi, W, D, rw, Hr, Wt);
            gtgt[pix] = fmaf(ls.f, gb - ga, ga);
        } else {
            gtgt[pix] = unwarp_sum(gtwx, b, x, row_shift(sv, W), ylo, yhi, W, D, rw, Hr, Wt);
        }
    }
}

// dS/ds(v) of the linear warp, one block per row: sum over u of the folded warped-target
// gradient times d tw(u)/ds = tgt(clamp(u + k)) - tgt(clamp(u + k + 1)), plus the add-back
// term sum_u dS/dl(u).  (The rounded warp has dS/ds = 0.)
__global__ void __launch_bounds__(256) k_dshift_grad(const float *__restrict__ gtwx, const float *__restrict__ tgt,
                                                     const float *__restrict__ shift,
                                                     const float *__restrict__ gdisp, float *__restrict__ gshift,
                                                     int W, int H, int D, int rw, int Hr, int Wt, int mode)
{
    __shared__ float red[8];
    const int y = blockIdx.x, b = blockIdx.y;
    float acc = 0.f;
    if (mode == STEREO_WARP_LINEAR) {
        const LinShift ls = lin_shift(shift[(size_t)b * H + y], W);
        const int ylo = y == 0 ? -rw : y, yhi = y == H - 1 ? H - 1 + rw : y;
        const float *trow = tgt + ((size_t)b * H + y) * W;
        const float *grow = gdisp + ((size_t)b * H + y) * W;
        for (int u = threadIdx.x; u < W; u += blockDim.x) {
            const float A = trow[clampi(u + ls.k, 0, W - 1)], B = trow[clampi(u + ls.k + 1, 0, W - 1)];
            acc = fmaf(fold_tw(gtwx, b, u, ylo, yhi, W, D, rw, Hr, Wt), A - B, acc);
            acc += grow[u];
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        gshift[(size_t)b * H + y] = t;
    }
}

// ------------------------------------------------------------------ launchers
template <int MODE, int RB>
cudaError_t launch_agg_rb(const AggArgs &a, int B, cudaStream_t st)
{
    constexpr int TW = agg_tx(MODE) + 2 * RB, TH = agg_ty(MODE) + 2 * RB;
    constexpr int NB = agg_dbuf(MODE) ? 2 : 1;
    const size_t smem = (size_t)TW * TH * (NB * sizeof(float4) * (kAggDC / 4) + sizeof(float)) +
                        (MODE == AGG_GC ? (size_t)kAggDC * agg_tx(MODE) * agg_ty(MODE) * sizeof(float) : 0);
    cudaError_t e = cudaFuncSetAttribute(k_dagg<MODE, RB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    dim3 grid((a.W + agg_tx(MODE) - 1) / agg_tx(MODE), (a.H + agg_ty(MODE) - 1) / agg_ty(MODE), B);
    k_dagg<MODE, RB><<<grid, agg_threads(MODE), smem, st>>>(a);
    return cudaGetLastError();
}

template <int MODE>
cudaError_t launch_agg(const AggArgs &a, int rb, int B, cudaStream_t st)
{
    switch (rb) {
    case 0: return launch_agg_rb<MODE, 0>(a, B, st);
    case 1: return launch_agg_rb<MODE, 1>(a, B, st);
    case 2: return launch_agg_rb<MODE, 2>(a, B, st);
    case 3: return launch_agg_rb<MODE, 3>(a, B, st);
    case 4: return launch_agg_rb<MODE, 4>(a, B, st);
    case 5: return launch_agg_rb<MODE, 5>(a, B, st);
    case 6: return launch_agg_rb<MODE, 6>(a, B, st);
    default: return launch_agg_rb<MODE, 7>(a, B, st);
    }
}

template <int RW>
cudaError_t launch_cb_rw(const CbArgs &a, int B, cudaStream_t st)
{
    constexpr int QW = 32 + 2 * RW, QH = kCbTY + 2 * RW, NP = 4 * kCbDC;
    const size_t smem = ((size_t)NP * ((QW | 1) * QH + 33 * QH + kCbTY * 32) + kCbTY * cb_diag_w(a.D)) * sizeof(float);
    cudaError_t e = cudaFuncSetAttribute(k_dcost_bwd<RW>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    dim3 grid((a.Wr + 31) / 32, (a.Hr + kCbTY - 1) / kCbTY, B);
    k_dcost_bwd<RW><<<grid, 256, smem, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_cb(const CbArgs &a, int rw, int B, cudaStream_t st)
{
    switch (rw) {
    case 0: return launch_cb_rw<0>(a, B, st);
    case 1: return launch_cb_rw<1>(a, B, st);
    case 2: return launch_cb_rw<2>(a, B, st);
    case 3: return launch_cb_rw<3>(a, B, st);
    case 4: return launch_cb_rw<4>(a, B, st);
    case 5: return launch_cb_rw<5>(a, B, st);
    case 6: return launch_cb_rw<6>(a, B, st);
    default: return launch_cb_rw<7>(a, B, st);
    }
}

AggArgs agg_args(const stereo_diff_params *p, const Dims &d, const Ws &w, const float *ref)
{
    AggArgs a;
    memset(&a, 0, sizeof(a));
    a.img = ref;
    a.W = d.W;
    a.H = d.H;
    a.D = d.D;
    a.warp_mode = d.warp_mode;
    a.kappa = sqrtf(kLog2e) / p->sigma1;
    a.k0 = -kLog2e / (p->sigma0 * p->sigma0);
    a.kT = kLog2e / p->temperature;
    a.invT = 1.0f / p->temperature;
    a.gw_scale = 2.0f / (p->sigma1 * p->sigma1 * a.kappa);
    a.lse = w.lse;
    a.lbar = w.lbar;
    return a;
}

}  // namespace
}  // namespace sgb

using namespace sgb;

extern "C" int stereo_diff_params_default(stereo_diff_params *p)
{
    if (!p) return set_error(STEREO_EINVAL, "stereo_diff_params_default: null pointer");
    memset(p, 0, sizeof(*p));
    p->batch = 1;
    p->win = 9;
    p->bil = 11;
    p->sigma0 = 1.5f;
    p->sigma1 = 5.5f;
    p->temperature = 0.1f;
    return STEREO_OK;
}

extern "C" int stereo_softargmin_workspace_bytes(const stereo_diff_params *p, size_t *bytes)
{
    Dims d;
    int rc = check_params(p, &d, "stereo_softargmin_workspace_bytes");
    if (rc) return rc;
    if (!bytes) return set_error(STEREO_EINVAL, "stereo_softargmin_workspace_bytes: null output");
    *bytes = layout(d, nullptr, nullptr);
    return STEREO_OK;
}

extern "C" int stereo_softargmin_fwd(const stereo_diff_params *p, const float *ref, const float *tgt,
                                     const float *shift, float *disp, void *ws, size_t ws_bytes,
                                     stereo_stream_t stream)
{
    static const char *who = "stereo_softargmin_fwd";
    Dims d;
    Ws w;
    int rc = check_params(p, &d, who);
    if (rc) return rc;
    if (!ref || !tgt || !shift || !disp) return set_error(STEREO_EINVAL, "%s: null pointer", who);
    if ((rc = check_ws(d, ws, ws_bytes, &w, who))) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    const int B = d.B;
    k_dwarp<<<dim3((d.W + 255) / 256, d.H, B), 256, 0, st>>>(tgt, shift, w.tw, d.W, d.H, d.warp_mode);
    const size_t ssm = (size_t)(32 + 2 * d.rw) * (8 + 2 * d.rw) * sizeof(float);
    launch_dstats(d.rw, dim3((d.W + 31) / 32, (d.H + 7) / 8, B), ssm, st, ref, d.W, d.H, d.W, 0, w.mur, w.sdr,
                  nullptr);
    launch_dstats(d.rw, dim3((d.We + 31) / 32, (d.H + 7) / 8, B), ssm, st, w.tw, d.W, d.H, d.We, -(d.D - 1), w.mut,
                  nullptr, w.isdt);
    const int nchunk = (d.D + kCostDC - 1) / kCostDC;
    const size_t csm = dcost_smem(d.rw);
    {
        const dim3 grid((d.W + kCostTX - 1) / kCostTX, (d.H + kCostTY - 1) / kCostTY, B * nchunk);
#define SGB_DCOST(R)                                                                                  \
    k_dcost<R><<<grid, kCostThreads, csm, st>>>(ref, w.tw, w.mur, w.sdr, w.mut, w.isdt, w.cost, d.W, d.H, d.D, nchunk)
        switch (d.rw) {
        case 0: SGB_DCOST(0); break;
        case 1: SGB_DCOST(1); break;
        case 2: SGB_DCOST(2); break;
        case 3: SGB_DCOST(3); break;
        case 4: SGB_DCOST(4); break;
        case 5: SGB_DCOST(5); break;
        case 6: SGB_DCOST(6); break;
        default: SGB_DCOST(7); break;
        }
#undef SGB_DCOST
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_error(e, who);
    AggArgs a = agg_args(p, d, w, ref);
    a.vol = w.cost;
    a.shift = shift;
    a.disp = disp;
    e = launch_agg<AGG_FWD>(a, d.rb, B, st);
    return cuda_error(e, who);
}

extern "C" int stereo_softargmin_bwd(const stereo_diff_params *p, const float *ref, const float *tgt,
                                     const float *shift, const float *gdisp, float *gref, float *gtgt,
                                     float *gshift, void *ws, size_t ws_bytes, stereo_stream_t stream)
{
    static const char *who = "stereo_softargmin_bwd";
    Dims d;
    Ws w;
    int rc = check_params(p, &d, who);
    if (rc) return rc;
    if (!ref || !tgt || !shift || !gdisp) return set_error(STEREO_EINVAL, "%s: null pointer", who);
    if ((rc = check_ws(d, ws, ws_bytes, &w, who))) return rc;
    if (!gref && !gtgt && !gshift) return STEREO_OK;
    cudaStream_t st = (cudaStream_t)stream;
    const int B = d.B;
    AggArgs a = agg_args(p, d, w, ref);
    a.vol = w.cost;
    a.gdisp = gdisp;
    a.h = w.h;
    a.beta = w.beta;
    a.t1 = w.t1;
    cudaError_t e = launch_agg<AGG_H>(a, d.rb, B, st);
    if (e != cudaSuccess) return cuda_error(e, who);
    a.vol = w.h;
    a.gc = w.gc;
    a.cost = w.cost;
    a.gw = w.gw;
    e = launch_agg<AGG_GC>(a, d.rb, B, st);
    if (e != cudaSuccess) return cuda_error(e, who);
    CbArgs c;
    c.ref = ref;
    c.tw = w.tw;
    c.mur = w.mur;
    c.sdr = w.sdr;
    c.mut = w.mut;
    c.isdt = w.isdt;
    c.cost = w.cost;
    c.gc = w.gc;
    const bool need_tw = gtgt || gshift;    // the warped-target gradient feeds both
    c.gpart = need_tw ? w.gpart : nullptr;
    c.grefx = w.grefx;
    c.W = d.W;
    c.H = d.H;
    c.D = d.D;
    c.Wr = d.Wr;
    c.Hr = d.Hr;
    c.We = d.We;
    c.inv_n = 1.0f / (float)d.n;
    if ((e = launch_cb(c, d.rw, B, st)) != cudaSuccess) return cuda_error(e, who);
    if (need_tw)
        k_dtgt_diag<<<dim3((d.Wt + 255) / 256, d.Hr, B), 256, 0, st>>>(w.gpart, w.gtwx, d.D, d.Wr, d.Hr, d.Wt);
    if (gref || gtgt)
        k_dfold<<<dim3((d.W + 255) / 256, d.H, B), 256, 0, st>>>(w.grefx, w.gw, w.gtwx, shift, gref, gtgt, d.W,
                                                                 d.H, d.D, d.rw, d.Wr, d.Hr, d.Wt, d.warp_mode);
    if (gshift)
        k_dshift_grad<<<dim3(d.H, B), 256, 0, st>>>(w.gtwx, tgt, shift, gdisp, gshift, d.W, d.H, d.D, d.rw, d.Hr,
                                                   d.Wt, d.warp_mode);
    return cuda_error(cudaGetLastError(), who);
}
