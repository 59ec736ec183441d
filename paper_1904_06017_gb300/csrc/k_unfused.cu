// k_unfused.cu -- the stage-per-kernel form of §3.2 with FP32 volumes in device memory:
// cost volume (eq. c), bilateral aggregation (eq. fbs), WTA + eq. (subpixel).
// Plain one-thread-per-pixel kernels; they read the staging buffers of k_prep.
#include "internal.cuh"

namespace sgb {

// eq. (c) for one pixel and every d: c = 1 - (n S - S_ref S_tar) / sqrt(A_ref A_tar),
// S the w x w correlation sum (exact integer), A = n sum I^2 - (sum I)^2.
__global__ void k_cost_volume(const uint8_t *__restrict__ ref_pad, const uint8_t *__restrict__ tgt_pad,
                              const int2 *__restrict__ ref_stats, const int2 *__restrict__ tgt_stats,
                              int W, int H, int D, int rw, int n, int pad_left, int pad_top,
                              int pad_w, int pad_pitch, float *__restrict__ cost)
{
    const int u = blockIdx.x * blockDim.x + threadIdx.x, v = blockIdx.y;
    if (u >= W || v >= H) return;
    const int px = u + pad_left, py = v + pad_top;
    const int2 r = ref_stats[(size_t)py * pad_w + px];
    float *out = cost + ((size_t)v * W + u) * D;
    for (int d = 0; d < D; ++d) {
        int S = 0;
        for (int dy = -rw; dy <= rw; ++dy) {
            const uint8_t *a = ref_pad + (size_t)(py + dy) * pad_pitch + px;
            const uint8_t *b = tgt_pad + (size_t)(py + dy) * pad_pitch + px - d;
            for (int dx = -rw; dx <= rw; ++dx) S += (int)a[dx] * (int)b[dx];
        }
        const int2 t = tgt_stats[(size_t)py * pad_w + px - d];
        const int num = n * S - r.x * t.x;
        out[d] = fmaf(-(float)num, __int_as_float(r.y) * __int_as_float(t.y), 1.0f);
    }
}

int launch_cost_volume(stereo_ctx *ctx, float *cost, cudaStream_t s)
{
    const Geometry &g = ctx->g;
    dim3 block(128), grid((g.W + 127) / 128, g.H);
    k_cost_volume<<<grid, block, 0, s>>>(ctx->ref_pad, ctx->tgt_pad, ctx->ref_stats, ctx->tgt_stats,
                                         g.W, g.H, g.D, g.rw, g.n, g.pad_left, g.pad_top, g.pad_w,
                                         g.pad_pitch, cost);
    return cuda_error(cudaGetLastError(), "k_cost_volume launch");
}

// eq. (fbs): E(p,d) = sum_q w(p,q) c(q,d) / sum_q w(p,q), q over the in-image part of
// the k x k window, w per eq. (omega_s) in FP32.  16 disparities per register chunk.
constexpr int kAggChunk = 16;

__global__ void k_aggregate_volume(const uint8_t *__restrict__ ref, int pitch, const float *__restrict__ cost,
                                   int W, int H, int D, int rb, float inv_s0sq, float inv_s1sq,
                                   float *__restrict__ agg)
{
    const int u = blockIdx.x * blockDim.x + threadIdx.x, v = blockIdx.y;
    if (u >= W || v >= H) return;
    const float Ip = ref[(size_t)v * pitch + u];
    float ws = 0.f;
    for (int dy = -rb; dy <= rb; ++dy)
        for (int dx = -rb; dx <= rb; ++dx) {
            const int uq = u + dx, vq = v + dy;
            if (uq < 0 || uq >= W || vq < 0 || vq >= H) continue;
            const float di = Ip - (float)ref[(size_t)vq * pitch + uq];
            ws += expf(-(float)(dx * dx + dy * dy) * inv_s0sq - di * di * inv_s1sq);
        }
    const float inv_ws = 1.0f / ws;
    for (int d0 = 0; d0 < D; d0 += kAggChunk) {
        float acc[kAggChunk];
#pragma unroll
        for (int k = 0; k < kAggChunk; ++k) acc[k] = 0.f;
        for (int dy = -rb; dy <= rb; ++dy)
            for (int dx = -rb; dx <= rb; ++dx) {
                const int uq = u + dx, vq = v + dy;
                if (uq < 0 || uq >= W || vq < 0 || vq >= H) continue;
                const float di = Ip - (float)ref[(size_t)vq * pitch + uq];
                const float w = expf(-(float)(dx * dx + dy * dy) * inv_s0sq - di * di * inv_s1sq);
                const float *cq = cost + ((size_t)vq * W + uq) * D + d0;
#pragma unroll
                for (int k = 0; k < kAggChunk; ++k)
                    if (d0 + k < D) acc[k] = fmaf(w, cq[k], acc[k]);
            }
        float *out = agg + ((size_t)v * W + u) * D + d0;
#pragma unroll
        for (int k = 0; k < kAggChunk; ++k)
            if (d0 + k < D) out[k] = acc[k] * inv_ws;
    }
}

int launch_aggregate_volume(stereo_ctx *ctx, const uint8_t *ref, const float *cost, float *agg,
                            cudaStream_t s)
{
    const Geometry &g = ctx->g;
    const float s0 = ctx->p.sigma0, s1 = ctx->p.sigma1;
    dim3 block(128), grid((g.W + 127) / 128, g.H);
    k_aggregate_volume<<<grid, block, 0, s>>>(ref, g.pitch, cost, g.W, g.H, g.D, g.rb, 1.0f / (s0 * s0),
                                              1.0f / (s1 * s1), agg);
    return cuda_error(cudaGetLastError(), "k_aggregate_volume launch");
}

// WTA (lowest d wins ties) + eq. (subpixel) on E, add back s_i(v) = floor(s(v) + 0.5).
__global__ void k_wta_volume(const float *__restrict__ agg, const float *__restrict__ shift, int W, int H,
                             int D, float *__restrict__ disp, int32_t *__restrict__ wta,
                             float *__restrict__ best2)
{
    const int u = blockIdx.x * blockDim.x + threadIdx.x, v = blockIdx.y;
    if (u >= W || v >= H) return;
    const float *e = agg + ((size_t)v * W + u) * D;
    int b = 0;
    for (int d = 1; d < D; ++d)
        if (e[d] < e[b]) b = d;
    float second = __int_as_float(0x7f800000);
    for (int d = 0; d < D; ++d)
        if (d != b && e[d] < second) second = e[d];
    float delta = 0.f;
    if (b > 0 && b < D - 1) {
        const float den = 2.f * e[b - 1] + 2.f * e[b + 1] - 4.f * e[b];
        if (den > 0.f) delta = (e[b - 1] - e[b + 1]) / den;
    }
    const int si = (int)floor((double)shift[v] + 0.5);
    const size_t o = (size_t)v * W + u;
    disp[o] = (float)b + delta + (float)si;
    if (wta) wta[o] = b;
    if (best2) {
        best2[2 * o] = e[b];
        best2[2 * o + 1] = second;
    }
}

int launch_wta_volume(stereo_ctx *ctx, const float *agg, const float *shift, float *disp,
                      int32_t *wta, float *best2, cudaStream_t s)
{
    const Geometry &g = ctx->g;
    dim3 block(128), grid((g.W + 127) / 128, g.H);
    k_wta_volume<<<grid, block, 0, s>>>(agg, shift, g.W, g.H, g.D, disp, wta, best2);
    return cuda_error(cudaGetLastError(), "k_wta_volume launch");
}

}  // namespace sgb
