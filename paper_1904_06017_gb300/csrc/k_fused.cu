// k_fused.cu -- fused matching cost (eq. c) + bilateral aggregation (eq. omega_s,
// eq. fbs) + winner-take-all + parabola sub-pixel step (eq. subpixel), §3.2.
//
// One CTA (8 warps) owns a 64 x 32 block of output pixels and all D disparities:
//  1. TMA (cp.async.bulk.tensor) stages the reference tile and the warped-target strip
//     (replicate-padded copies) into shared memory, one box each, on an mbarrier.
//  2. For each chunk of DC disparities:
//     a. vertical running sums of the products I_ref(x,y) I_tar(x-d,y) over the w rows
//        of the block (exact integers), one walker per (column, d);
//     b. horizontal running sums of those (the full w x w correlation sum of eq. c),
//        then c = 1 - (n S - S_ref S_tar) / sqrt(A_ref A_tar), written in place: the
//        chunk's cost volume for the tile plus its bilateral halo lives only in shared
//        memory, never in device memory;
//     c. aggregation: each thread owns a column of kPY pixels x DC disparities in
//        registers; for every neighbour row it loads the DC costs once (LDS.128) and
//        applies them to every pixel whose window holds it, with the weight
//        w = 2^(K[dx][dy] - (s I_q - s I_p)^2) (eq. omega0 x eq. omega1 in one base-2
//        exponent, MUFU ex2) and packed f32x2 FMAs over pairs of disparities;
//     d. running WTA over d (lowest d wins ties) keeping the neighbours of the best d.
//  3. Epilogue: eq. (subpixel) on the winner's neighbours, add back s_i(v), write.
// Normalising by sum_q w(p,q) is skipped: it is a positive per-pixel constant, so the
// argmin and the (scale-free) parabola step do not change.
#include "internal.cuh"

namespace sgb {

struct FusedArgs {
    const int2 *ref_stats;
    const int2 *tgt_stats;
    const float *shift;
    float *disp;
    int32_t *wta;
    uint8_t *valid;
    int *status;
    int W, H, D, Dp, rw, m, n;
    int pad_left, pad_top, pad_w;
    int ref_e, tgt_e, ref_box_w, tgt_box_w, box_h, ref_box_x;
    float iscale;
    float K[(2 * kMaxRB + 1) * (2 * kMaxRB + 1)];
};

__host__ __device__ constexpr size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// ----------------------------------------------------------------- PTX helpers
__device__ __forceinline__ uint32_t smem_addr(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, int c0, int c1,
                                            int c2, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_addr(dst)),
        "l"(map), "r"(c0), "r"(c1), "r"(c2), "r"(smem_addr(bar))
        : "memory");
}

__device__ __forceinline__ float ex2_approx(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Shared-memory layout (all offsets from the dynamic base, which is 128-byte aligned).
struct SmemLayout {
    size_t sref, stgt, cbuf, sI, sK, bar, flag, total;
};

__host__ __device__ inline SmemLayout smem_layout(int rb, int m, int dc, int ref_box_w,
                                                  int tgt_box_w, int box_h)
{
    SmemLayout L;
    const int QH = kTileY + 2 * rb, QW = kTileX + 2 * rb, CW = kTileX + 2 * m, KB = 2 * rb + 1;
    L.sref = 0;
    L.stgt = align_up(L.sref + (size_t)box_h * ref_box_w, 128);
    L.cbuf = align_up(L.stgt + (size_t)box_h * tgt_box_w, 128);
    L.sI = align_up(L.cbuf + (size_t)QH * CW * dc * 4, 16);
    L.sK = align_up(L.sI + (size_t)QH * QW * 4, 16);
    L.bar = align_up(L.sK + (size_t)KB * KB * 4, 8);
    L.flag = L.bar + 8;
    L.total = align_up(L.flag + 8, 128);
    return L;
}

size_t fused_smem_bytes(const Geometry &g)
{
    return smem_layout(g.rb, g.m, g.dc, g.ref_box_w, g.tgt_box_w, g.box_h).total;
}

template <int RB, int DC>
__global__ void __launch_bounds__(kThreads, 1)
k_fused(const __grid_constant__ CUtensorMap tmap_ref, const __grid_constant__ CUtensorMap tmap_tgt,
        const __grid_constant__ FusedArgs a)
{
    static_assert(DC % 4 == 0, "DC must be a multiple of 4");
    constexpr int KB = 2 * RB + 1;
    constexpr int QH = kTileY + 2 * RB, QW = kTileX + 2 * RB;
    constexpr int NR = kPY + 2 * RB;   // neighbour rows seen by one thread's pixel column
    extern __shared__ __align__(128) uint8_t smem[];

    const int CW = kTileX + 2 * a.m;
    const int RP = a.ref_box_w, TP = a.tgt_box_w;
    const SmemLayout L = smem_layout(RB, a.m, DC, RP, TP, a.box_h);
    uint8_t *sref = smem + L.sref;
    uint8_t *stgt = smem + L.stgt;
    float *cbuf = reinterpret_cast<float *>(smem + L.cbuf);
    float *sI = reinterpret_cast<float *>(smem + L.sI);
    float *sK = reinterpret_cast<float *>(smem + L.sK);
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + L.bar);
    int *flag = reinterpret_cast<int *>(smem + L.flag);

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int x0 = blockIdx.x * kTileX, y0 = blockIdx.y * kTileY;

    // ---- 1. stage the image tiles with TMA
    if (tid == 0) mbar_init(bar, 1);
    for (int i = tid; i < KB * KB; i += kThreads) sK[i] = a.K[i];
    __syncthreads();
    if (tid == 0) {
        mbar_expect_tx(bar, (uint32_t)(a.box_h * (RP + TP)));
        tma_load_3d(sref, &tmap_ref, 0, (x0 + a.ref_box_x) / 16, y0, bar);
        tma_load_3d(stgt, &tmap_tgt, 0, x0 / 16, y0, bar);
        // bounded wait (about a second of clock cycles), then give up with a status flag
        const long long t0 = clock64();
        bool ok = false;
        while (!(ok = mbar_try_wait(bar, 0)) && clock64() - t0 < (1ll << 31)) {
        }
        *flag = ok ? 1 : 0;
        if (!ok) atomicOr(a.status, 1);
    }
    __syncthreads();
    if (*flag == 0) return;

    const int rw = a.rw, wsz = 2 * rw + 1;
    // scaled reference intensities of the cost positions (tile + bilateral halo); a
    // position outside the image gets a huge value so its weight underflows to 0
    for (int i = tid; i < QH * QW; i += kThreads) {
        const int yq = i / QW, xq = i - yq * QW;
        const int ix = x0 - RB + xq, iy = y0 - RB + yq;
        float v = 1e18f;
        if (ix >= 0 && ix < a.W && iy >= 0 && iy < a.H)
            v = (float)sref[(yq + rw) * RP + a.ref_e + xq + rw] * a.iscale;
        sI[i] = v;
    }
    __syncthreads();

    const int xt = (warp & 1) * 32 + lane;
    const int yt0 = (warp >> 1) * kPY;
    float Ip[kPY];
#pragma unroll
    for (int i = 0; i < kPY; ++i) Ip[i] = sI[(yt0 + i + RB) * QW + xt + RB];

    float best[kPY], bm1[kPY], bp1[kPY], prev[kPY];
    int bd[kPY];
#pragma unroll
    for (int i = 0; i < kPY; ++i) {
        best[i] = __int_as_float(0x7f800000);
        bm1[i] = bp1[i] = prev[i] = best[i];
        bd[i] = -1;
    }

    const size_t rowstride = (size_t)CW * DC;
    for (int d0 = 0; d0 < a.D; d0 += DC) {
        // ---- 2a. vertical sums of products, one walker per (product column, d)
        for (int w = tid; w < CW * DC; w += kThreads) {
            const int xp = w / DC, dd = w - xp * DC;
            const uint8_t *rc = sref + a.ref_e + xp;
            const uint8_t *tc = stgt + a.tgt_e + xp + (a.Dp - 1) - (d0 + dd);
            int acc = 0;
            for (int i = 0; i < wsz; ++i) acc += (int)rc[i * RP] * (int)tc[i * TP];
            int *o = reinterpret_cast<int *>(cbuf) + xp * DC + dd;
            o[0] = acc;
            for (int yq = 1; yq < QH; ++yq) {
                const int ya = yq + wsz - 1, yr = yq - 1;
                acc += (int)rc[ya * RP] * (int)tc[ya * TP] - (int)rc[yr * RP] * (int)tc[yr * TP];
                o[yq * rowstride] = acc;
            }
        }
        __syncthreads();
        // ---- 2b. horizontal sums and the cost of eq. (c), in place
        for (int w = tid; w < QH * DC; w += kThreads) {
            const int yq = w / DC, dd = w - yq * DC;
            const int d = d0 + dd;
            int *row = reinterpret_cast<int *>(cbuf) + yq * rowstride + dd;
            int S = 0;
            for (int j = 0; j < wsz; ++j) S += row[j * DC];
            const size_t prow = (size_t)(y0 - RB + yq + a.pad_top) * a.pad_w;
            const int pcol = x0 - RB + a.pad_left;
            const int2 *rs = a.ref_stats + prow + pcol;
            const int2 *ts = a.tgt_stats + prow + pcol - d;
            for (int xq = 0; xq < QW; ++xq) {
                const int vold = row[xq * DC];
                const int2 r = __ldg(rs + xq), t = __ldg(ts + xq);
                const int num = a.n * S - r.x * t.x;
                const float c = fmaf(-(float)num, __int_as_float(r.y) * __int_as_float(t.y), 1.0f);
                reinterpret_cast<float *>(row)[xq * DC] = c;
                if (xq + 1 < QW) S += row[(xq + wsz) * DC] - vold;
            }
        }
        __syncthreads();
        // ---- 2c. bilateral aggregation of the chunk
        float2 acc[kPY][DC / 2];
#pragma unroll
        for (int i = 0; i < kPY; ++i)
#pragma unroll
            for (int k = 0; k < DC / 2; ++k) acc[i][k] = make_float2(0.f, 0.f);
        for (int dx = 0; dx < KB; ++dx) {
            float Kr[KB];
#pragma unroll
            for (int j = 0; j < KB; ++j) Kr[j] = sK[dx * KB + j];
            const float *cb = cbuf + ((size_t)yt0 * CW + xt + dx) * DC;
            const float *ib = sI + yt0 * QW + xt + dx;
#pragma unroll
            for (int r = 0; r < NR; ++r) {
                const float4 *c4 = reinterpret_cast<const float4 *>(cb + r * rowstride);
                float4 q[DC / 4];
#pragma unroll
                for (int k = 0; k < DC / 4; ++k) q[k] = c4[k];
                const float Iq = ib[r * QW];
#pragma unroll
                for (int i = 0; i < kPY; ++i) {
                    const int dy = r - i;          // neighbour row - pixel row + RB
                    if (dy < 0 || dy > 2 * RB) continue;
                    const float t = Iq - Ip[i];
                    const float wgt = ex2_approx(fmaf(-t, t, Kr[dy]));
                    const float2 w2 = make_float2(wgt, wgt);
#pragma unroll
                    for (int k = 0; k < DC / 4; ++k) {
                        acc[i][2 * k] = __ffma2_rn(w2, make_float2(q[k].x, q[k].y), acc[i][2 * k]);
                        acc[i][2 * k + 1] = __ffma2_rn(w2, make_float2(q[k].z, q[k].w), acc[i][2 * k + 1]);
                    }
                }
            }
        }
        // ---- 2d. running WTA over the chunk, lowest d first
#pragma unroll
        for (int i = 0; i < kPY; ++i)
#pragma unroll
            for (int dd = 0; dd < DC; ++dd) {
                const int d = d0 + dd;
                if (d >= a.D) break;
                const float v = (dd & 1) ? acc[i][dd >> 1].y : acc[i][dd >> 1].x;
                if (v < best[i]) {
                    best[i] = v;
                    bd[i] = d;
                    bm1[i] = prev[i];
                } else if (d == bd[i] + 1) {
                    bp1[i] = v;
                }
                prev[i] = v;
            }
        __syncthreads();
    }

    // ---- 3. epilogue: eq. (subpixel), add back s_i(v)
#pragma unroll
    for (int i = 0; i < kPY; ++i) {
        const int u = x0 + xt, v = y0 + yt0 + i;
        if (u >= a.W || v >= a.H) continue;
        const int si = (int)floor((double)__ldg(a.shift + v) + 0.5);
        float delta = 0.f;
        if (bd[i] > 0 && bd[i] < a.D - 1) {
            const float den = 2.f * bm1[i] + 2.f * bp1[i] - 4.f * best[i];
            if (den > 0.f) delta = (bm1[i] - bp1[i]) / den;
        }
        const size_t o = (size_t)v * a.W + u;
        a.disp[o] = (float)bd[i] + delta + (float)si;
        if (a.wta) a.wta[o] = bd[i];
        if (a.valid) {
            int s_hi = -(1 << 30), s_lo = 1 << 30;
            for (int y = max(v - a.m, 0); y <= min(v + a.m, a.H - 1); ++y) {
                const int s = (int)floor((double)__ldg(a.shift + y) + 0.5);
                s_hi = max(s_hi, s);
                s_lo = min(s_lo, s);
            }
            const int ulo = a.m + a.D - 1 + max(0, s_hi);
            const int uhi = a.W - 1 - a.m + min(0, s_lo);
            a.valid[o] = (uint8_t)(v >= a.m && v <= a.H - 1 - a.m && u >= ulo && u <= uhi);
        }
    }
}

typedef void (*FusedKernel)(const CUtensorMap, const CUtensorMap, const FusedArgs);

template <int DC>
static FusedKernel pick_rb(int rb)
{
    switch (rb) {
    case 0: return k_fused<0, DC>;
    case 1: return k_fused<1, DC>;
    case 2: return k_fused<2, DC>;
    case 3: return k_fused<3, DC>;
    case 4: return k_fused<4, DC>;
    case 5: return k_fused<5, DC>;
    case 6: return k_fused<6, DC>;
    case 7: return k_fused<7, DC>;
    }
    return nullptr;
}

static FusedKernel pick(const Geometry &g)
{
    if (g.dc == 12) return pick_rb<12>(g.rb);
    if (g.dc == 4) return pick_rb<4>(g.rb);
    return nullptr;
}

int fused_configure(stereo_ctx *ctx)
{
    FusedKernel k = pick(ctx->g);
    if (!k) return set_error(STEREO_ENOTSUP, "no fused kernel for bil=%d dc=%d", ctx->p.bil, ctx->g.dc);
    return cuda_error(cudaFuncSetAttribute((const void *)k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)ctx->g.smem_bytes),
                      "cudaFuncSetAttribute(fused)");
}

int launch_fused(stereo_ctx *ctx, const float *shift, float *disp, int32_t *wta, uint8_t *valid,
                 cudaStream_t s)
{
    const Geometry &g = ctx->g;
    FusedKernel k = pick(g);
    if (!k) return set_error(STEREO_ENOTSUP, "no fused kernel for bil=%d", ctx->p.bil);
    FusedArgs a;
    a.ref_stats = ctx->ref_stats;
    a.tgt_stats = ctx->tgt_stats;
    a.shift = shift;
    a.disp = disp;
    a.wta = wta;
    a.valid = valid;
    a.status = ctx->status_dev;
    a.W = g.W;
    a.H = g.H;
    a.D = g.D;
    a.Dp = g.Dp;
    a.rw = g.rw;
    a.m = g.m;
    a.n = g.n;
    a.pad_left = g.pad_left;
    a.pad_top = g.pad_top;
    a.pad_w = g.pad_w;
    a.ref_e = g.ref_e;
    a.tgt_e = g.tgt_e;
    a.ref_box_w = g.ref_box_w;
    a.tgt_box_w = g.tgt_box_w;
    a.box_h = g.box_h;
    a.ref_box_x = g.pad_left - (int)align_up(g.m, 16);
    a.iscale = ctx->iscale;
    const int kb = 2 * g.rb + 1;
    for (int i = 0; i < kb * kb; ++i) a.K[i] = ctx->kspatial[i];
    dim3 grid(g.ntx, g.nty);
    k<<<grid, kThreads, g.smem_bytes, s>>>(ctx->tmap_ref, ctx->tmap_tgt, a);
    return cuda_error(cudaGetLastError(), "k_fused launch");
}

}  // namespace sgb
