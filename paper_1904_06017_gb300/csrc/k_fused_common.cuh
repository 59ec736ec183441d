// k_fused_common.cuh -- what the fused kernels share: their arguments and pair descriptors,
// the PTX helpers (mbarrier, TMA), tile claiming and staging, cost storage types, the
// shared-memory layout of the FP32-layout kernels, and the kernel-choice declarations.
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <type_traits>
#include <utility>

#include "internal.cuh"

namespace sgb {

struct FusedArgs {
    const int2 *ref_stats;
    const int2 *tgt_stats;
    const int4 *row_tab;
    float *disp;
    int32_t *wta;
    uint8_t *valid;
    float *best2;       // optional [H][W][2]: normalised E at d* and the smallest E over d != d*
    int *status;
    int stall_test;     // test hook: arm the staging barrier but issue no copy (the wait expires)
    int W, H, D, Dp, rw, m, n;
    int pad_left, pad_top, pad_w;
    int ref_e, tgt_e, ref_box_w, tgt_box_w, box_h, ref_box_x;
    float iscale;
    float K[(2 * kMaxRB + 1) * (2 * kMaxRB + 1)];
};

// Everything one pair needs: its two tensor maps (replicate-padded reference and warped
// target) and its arguments.  A single-pair launch passes one as a __grid_constant__
// parameter; a batch passes a device array of them.
struct PairDesc {
    CUtensorMap tmap_ref;
    CUtensorMap tmap_tgt;
    FusedArgs a;
    int ntx, nty;   // tiles in x and y
};

constexpr int kBand = 6;   // cost rows per band of the two-pass window sums
constexpr int kSeg = 5;    // cost columns per horizontal-pass work item (5: conflict-free LDS.128 strides)

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

// ----------------------------------------------------------------- tile claim and staging
// Claims the launch's next tile: a single pair walks its tiles in a fixed order (blockIdx.x,
// + gridDim.x, ...); a batch claims work-list items (pair, tile) with an atomic counter,
// heaviest first.  Copies the tile's pair arguments to s_args and returns its descriptor, or
// nullptr once the work list is exhausted.  Called by all NT threads of the CTA.
template <int NT>
__device__ __forceinline__ const PairDesc *claim_tile(const PairDesc &single, const PairDesc *pairs,
                                                      const int2 *items, int nitems, int *counter, int iter,
                                                      FusedArgs &s_args, int &s_item, int tid, int &tx, int &ty)
{
    if (tid == 0) s_item = pairs ? atomicAdd(counter, 1) : (int)blockIdx.x + iter * (int)gridDim.x;
    __syncthreads();
    const int item = s_item;
    if (item >= nitems) return nullptr;
    int p = 0;
    if (pairs) {
        const int2 it = items[item];
        p = it.x;
        tx = it.y & 0xffff;
        ty = it.y >> 16;
    } else {
        tx = item % single.ntx;
        ty = item / single.ntx;
    }
    const PairDesc *pd = pairs ? pairs + p : &single;
    const int *src = reinterpret_cast<const int *>(&pd->a);
    int *dst = reinterpret_cast<int *>(&s_args);
    for (int i = tid; i < (int)(sizeof(FusedArgs) / 4); i += NT) dst[i] = src[i];
    __syncthreads();
    return pd;
}

// Stages the reference tile and the warped-target strip of the tile at (x0, y0) into sref /
// stgt with TMA; the mbarrier completes once per tile (phase iter & 1).  The wait is bounded
// (about a second of clock cycles): false, with the status word set, when the copies did not
// land.  That limit is a fail-safe that should never fire: when it does, the CTA returns and
// its copies may still be in flight into its shared memory, and the launch's outputs are
// invalid (the host reads the status word with stereo_check_device_status, which reports
// STEREO_ETIMEOUT).  With the test hook stall_test set, thread 0 arms the barrier's
// transaction count but issues no copy, so nothing is in flight when the wait expires (after
// about a millisecond): the failure path then runs on purpose, without any fault.  The
// caller's barrier before this call orders the previous tile's shared-memory accesses before
// the copies that overwrite the same bytes.
__device__ __forceinline__ bool stage_images(const PairDesc *pd, const FusedArgs &a, uint8_t *sref, uint8_t *stgt,
                                             uint64_t *bar, int *flag, int x0, int y0, int iter, int tid)
{
    if (tid == 0) {
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_expect_tx(bar, (uint32_t)(a.box_h * (a.ref_box_w + a.tgt_box_w)));
        const bool stall = a.stall_test != 0;
        if (!stall) {
            tma_load_3d(sref, &pd->tmap_ref, 0, (x0 + a.ref_box_x) / 16, y0, bar);
            tma_load_3d(stgt, &pd->tmap_tgt, 0, x0 / 16, y0, bar);
        }
        const long long limit = stall ? (1ll << 21) : (1ll << 31);
        const long long t0 = clock64();
        bool ok = false;
        while (!(ok = mbar_try_wait(bar, (uint32_t)(iter & 1))) && clock64() - t0 < limit) {
        }
        *flag = ok ? 1 : 0;
        if (!ok) atomicOr(a.status, 1);
    }
    __syncthreads();
    return *flag != 0;
}

// Cost storage in shared memory: FP32, or FP16 / BF16 (rounded to nearest, widened back to
// FP32 when loaded; aggregation always accumulates in FP32).  store4 writes the costs of
// four consecutive disparities; load4 reads them back as two float2 pairs.
template <typename T> struct CostStore;
template <> struct CostStore<float> {
    static __device__ __forceinline__ void store4(float *p, float4 c) { *reinterpret_cast<float4 *>(p) = c; }
    static __device__ __forceinline__ void load4(const float *p, float2 &a, float2 &b)
    {
        const float4 v = *reinterpret_cast<const float4 *>(p);
        a = make_float2(v.x, v.y);
        b = make_float2(v.z, v.w);
    }
};
template <> struct CostStore<__half> {
    static __device__ __forceinline__ void store4(__half *p, float4 c)
    {
        uint32_t lo, hi;
        asm("cvt.rn.f16x2.f32 %0, %1, %2;" : "=r"(lo) : "f"(c.y), "f"(c.x));
        asm("cvt.rn.f16x2.f32 %0, %1, %2;" : "=r"(hi) : "f"(c.w), "f"(c.z));
        *reinterpret_cast<uint2 *>(p) = make_uint2(lo, hi);
    }
    static __device__ __forceinline__ void load4(const __half *p, float2 &a, float2 &b)
    {
        const uint2 v = *reinterpret_cast<const uint2 *>(p);
        a = __half22float2(*reinterpret_cast<const __half2 *>(&v.x));
        b = __half22float2(*reinterpret_cast<const __half2 *>(&v.y));
    }
};
template <> struct CostStore<__nv_bfloat16> {
    static __device__ __forceinline__ void store4(__nv_bfloat16 *p, float4 c)
    {
        uint32_t lo, hi;
        asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(lo) : "f"(c.y), "f"(c.x));
        asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(hi) : "f"(c.w), "f"(c.z));
        *reinterpret_cast<uint2 *>(p) = make_uint2(lo, hi);
    }
    // a BF16 value is the top half of its FP32: byte moves only (no arithmetic pipe)
    static __device__ __forceinline__ float lo_f(uint32_t w) { return __int_as_float(__byte_perm(w, 0, 0x1044)); }
    static __device__ __forceinline__ float hi_f(uint32_t w) { return __int_as_float(w & 0xffff0000u); }
    static __device__ __forceinline__ void load4(const __nv_bfloat16 *p, float2 &a, float2 &b)
    {
        const uint2 v = *reinterpret_cast<const uint2 *>(p);
        a = make_float2(lo_f(v.x), hi_f(v.x));
        b = make_float2(lo_f(v.y), hi_f(v.y));
    }
};

// Shared-memory layout (offsets from the dynamic base, which is 128-byte aligned):
//   sref  [box_h][ref_box_w] u8     reference tile (TMA)
//   stgt  [box_h][tgt_box_w] u8     warped-target strip (TMA)
//   cbuf  [QH][QW][DC] f32          the chunk's costs at the tile + bilateral halo
//   vband [kBand][CW][DC] i32       vertical window sums of one band of cost rows
//   sstr  [kBand][QW] int2          window statistics of the reference, this band
//   sstt  [kBand][QW+DC-1] int2     window statistics of the target behind the band's costs
//   sI    [QH][QW] f32              scaled reference intensity at the cost positions
//   sK    [KB][KB] f32              spatial part of the weight exponent
struct SmemLayout {
    size_t sref, stgt, cbuf, cbuf1, vband, sstr, sstt, sI, sK, total;
};

// nbuf cost buffers (2 for the warp-specialised form), band cost rows per window-sum band;
// band = 0 for the tensor-core cost phase, which needs no vband / sstr / sstt.
__host__ __device__ inline SmemLayout smem_layout(int rb, int m, int dc, int ref_box_w,
                                                  int tgt_box_w, int box_h, int esize, int tx, int ty,
                                                  int nbuf = 1, int band = kBand)
{
    SmemLayout L;
    const int QH = ty + 2 * rb, QW = tx + 2 * rb, CW = tx + 2 * m, KB = 2 * rb + 1;
    const size_t cbytes = align_up((size_t)QH * QW * dc * esize, 128);
    L.sref = 0;
    L.stgt = align_up(L.sref + (size_t)box_h * ref_box_w, 128);
    L.cbuf = align_up(L.stgt + (size_t)box_h * tgt_box_w, 128);
    L.cbuf1 = L.cbuf + (nbuf > 1 ? cbytes : 0);
    L.vband = L.cbuf + (size_t)nbuf * cbytes;
    L.sstr = align_up(L.vband + (size_t)band * CW * dc * 4, 16);
    L.sstt = align_up(L.sstr + (size_t)band * QW * 8, 16);
    L.sI = align_up(L.sstt + (size_t)band * (QW + dc - 1) * 8, 16);   // band 0: vband = sstr = sstt = sI
    L.sK = align_up(L.sI + (size_t)QH * QW * 4, 16);
    L.total = align_up(L.sK + (size_t)KB * KB * 4, 128);
    return L;
}

typedef void (*FusedKernel)(const PairDesc, const PairDesc *, const int2 *, int, int *);

// Kernel choice by (bilateral radius, disparities per chunk, warp columns); one translation
// unit per storage type and tile family keeps the instantiations compiling in parallel.
FusedKernel pick_fused_f32(int rb, int dc, int wc);    // k_fused_f32.cu: WC = 2, DC in {12, 4}
FusedKernel pick_fused_f32_tiles(int rb, int dc, int wc);  // k_fused_f32_tiles.cu: WC in {1, 4}, DC = 12
FusedKernel pick_fused_f32_wc4(int rb);                // k_fused_f32_wc4.cu: WC = 4, DC = 12
FusedKernel pick_fused_f32_dc4(int rb);                // k_fused_f32_dc4.cu: WC = 2, DC = 4
FusedKernel pick_fused_f16(int rb, int dc, int wc);    // k_fused_f16.cu: WC = 2, DC = 12
FusedKernel pick_fused_bf16(int rb, int dc, int wc);   // k_fused_bf16.cu: WC = 2, DC = 12
FusedKernel pick_fused_ws(int rb, int dc);             // k_fused_ws.cu: warp-specialised, FP32, DC = 12
FusedKernel pick_fused_tc(int cost_dtype, int rb);     // k_fused_tc_{f16,bf16}.cu: tensor-core aggregation, DC = 16
FusedKernel pick_fused_sc(int rb);                     // k_fused_sc.cu: screened FP32 form, tile code kScWC
FusedKernel pick_fused_sc_b2(int rb);                  // k_fused_sc_b2.cu: the same with the best2 output
FusedKernel pick_fused_sc16(int cost_dtype, int rb);   // k_fused_sc16.cu: FP16 / BF16 storage, tile code kScWC
FusedKernel pick_fused_sc16_b2(int cost_dtype, int rb);   // k_fused_sc16_b2.cu: the same with best2
FusedKernel pick_fused(int cost_dtype, int rb, int dc, int wc);
// The instantiation with the best2 output (FP32 storage at WC = 2 with DC = 12, and the
// tensor-core form); nullptr where there is none.  k_fused_b2_f32.cu, k_fused_tc_{f16,bf16}_b2.cu.
FusedKernel pick_fused_b2(int cost_dtype, int rb, int dc, int wc);
FusedKernel pick_fused_f32_b2(int rb, int dc);
FusedKernel pick_fused_tc_b2(int cost_dtype, int rb);
// The descriptor of one context for one call (k_fused_f32.cu).
void fill_pair_desc(const stereo_ctx *ctx, float *disp, int32_t *wta, uint8_t *valid, PairDesc &d,
                    float *best2 = nullptr);

}  // namespace sgb
