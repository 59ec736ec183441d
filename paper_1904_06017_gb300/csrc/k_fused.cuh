// k_fused.cuh -- fused matching cost (eq. c) + bilateral aggregation (eq. omega_s,
// eq. fbs) + winner-take-all + parabola sub-pixel step (eq. subpixel), §3.2.
//
// One CTA of kWarps warps owns a block of output pixels (64 x 36 by default) and all D
// disparities; the kernel is persistent over tiles (and, for a batch, over pairs):
//  1. TMA (cp.async.bulk.tensor) stages the reference tile and the warped-target strip
//     (replicate-padded copies) into shared memory, one box each, on an mbarrier.
//  2. For each chunk of DC disparities, the chunk's costs at the tile plus its bilateral halo,
//     eq. (c), into shared memory (never device memory):
//     cost_chunk_mma (k_fused) -- the cross term sum I_ref I_tar of every block on the tensor
//        cores (exact FP16 operands, exact FP32 accumulation), one warp per 8-column block
//        walking down its rows with the window as a running sum in the accumulator;
//     cost_chunk (the warp-specialised form, and k_fused_tc.cuh) -- vertical running sums of
//        the products per (product column, d) and horizontal sums over the w columns, band
//        by band of cost rows;
//     then c = 1 - (n S - S_ref S_tar) / sqrt(A_ref A_tar) with exact integer numerators.
//  3. Aggregation: each thread owns a column of kPY pixels x DC disparities in registers;
//     for every neighbour row it loads the DC costs once (LDS.128, the next row prefetched)
//     and applies them to every pixel whose window holds it, with the weight
//     w = 2^(K[dx][dy] - (s I_q - s I_p)^2) (eq. omega0 x eq. omega1 in one base-2
//     exponent, MUFU ex2) and packed f32x2 FMAs over disparity pairs; then a running WTA
//     over d (lowest d wins ties) keeping the neighbours of the best d.
//  4. Epilogue: eq. (subpixel) on the winner's neighbours, add back s_i(v), write.
// Normalising by sum_q w(p,q) is skipped: it is a positive per-pixel constant, so the
// argmin and the (scale-free) parabola step do not change.
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
// land.  The caller's barrier before this call orders the previous tile's shared-memory
// accesses before the copies that overwrite the same bytes.
__device__ __forceinline__ bool stage_images(const PairDesc *pd, const FusedArgs &a, uint8_t *sref, uint8_t *stgt,
                                             uint64_t *bar, int *flag, int x0, int y0, int iter, int tid)
{
    if (tid == 0) {
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_expect_tx(bar, (uint32_t)(a.box_h * (a.ref_box_w + a.tgt_box_w)));
        tma_load_3d(sref, &pd->tmap_ref, 0, (x0 + a.ref_box_x) / 16, y0, bar);
        tma_load_3d(stgt, &pd->tmap_tgt, 0, x0 / 16, y0, bar);
        const long long t0 = clock64();
        bool ok = false;
        while (!(ok = mbar_try_wait(bar, (uint32_t)(iter & 1))) && clock64() - t0 < (1ll << 31)) {
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


// The costs of one chunk of DC disparities at the tile plus its bilateral halo (QH x QW
// positions), eq. (c), into cbuf[QH][QW][DC], band by band of kBand cost rows:
//  vertical pass: V(x, y, d) = sum_{i < w} I_ref(x, y+i) I_tar(x-d, y+i), one walker per
//      (product column x, d), a running sum carried in a register from band to band;
//  horizontal pass: S = sum_{j < w} V(x+j, y, d) for four d per work item, then
//      c = 1 - (n S - S_ref S_tar) r_ref r_tar with the staged window statistics.
// Every pass issues all of its shared-memory loads before its stores, so the loads of a
// band are in flight together instead of waiting behind stores they might alias.
// Synchronisation of the NT threads that run cost_chunk: the whole CTA (BAR = 0) or a named
// barrier BAR of NT threads (the producer warps of the warp-specialised form).
// Calls f(std::integral_constant<int, i>) for i = 0 .. N-1 (compile-time loop).
template <typename F, int... I>
__device__ __forceinline__ void static_for_impl(F &&f, std::integer_sequence<int, I...>)
{
    (f(std::integral_constant<int, I>{}), ...);
}
template <int N, typename F>
__device__ __forceinline__ void static_for(F &&f)
{
    static_for_impl(f, std::make_integer_sequence<int, N>{});
}

template <int BAR, int NT>
__device__ __forceinline__ void group_sync()
{
    if constexpr (BAR == 0) __syncthreads();
    else asm volatile("bar.sync %0, %1;" ::"n"(BAR), "n"(NT) : "memory");
}

template <int RB, int DC, int RW, typename T, int TX, int TY, int NT = kThreads, int BAR = 0,
          int KBAND = kBand, bool SWZ = false>
__device__ __forceinline__ void cost_chunk(const FusedArgs &a, const uint8_t *sref, const uint8_t *stgt,
                                           T *cbuf, int *vband, int2 *sstr, int2 *sstt,
                                           int x0, int y0, int d0, int tid)
{
    constexpr int kThreads = NT, kBand = KBAND;      // the threads and band of this instantiation
    constexpr int WS = 2 * RW + 1;                    // block size w
    constexpr int QH = TY + 2 * RB, QW = TX + 2 * RB;
    constexpr int CW = TX + 2 * (RW + RB);            // product columns
    constexpr int NQ = DC / 4;
    constexpr int NSEG = (QW + kSeg - 1) / kSeg;
    constexpr int NWV = (CW * DC + kThreads - 1) / kThreads;   // vertical walkers per thread
    constexpr int TSW = QW + DC - 1;                  // target-statistics columns of a chunk
    constexpr int NST = (kBand * (QW + TSW) + kThreads - 1) / kThreads;
    // the reference box pitch and column offset follow from the radii and the tile width
    // (the same formulas as the host's geometry); the target box depends on the search range
    constexpr int MM = RW + RB;
    constexpr int REFE = (MM + 15) / 16 * 16 - MM;
    constexpr int RP = (REFE + TX + 2 * MM + 15) / 16 * 16;
    const int TP = a.tgt_box_w;
    const size_t crow = (size_t)QW * DC;
    // The products I_ref I_tar of a walker live in a register ring of NPH * kBand slots, product
    // row j in slot j mod RING: the row entering a cost row's window is loaded once and read
    // back from the ring when it leaves, w rows later.  Bands cycle through the NPH phases of
    // the ring, so every slot index is a compile-time constant.
    constexpr int NPH = (WS + 1 + kBand - 1) / kBand;
    constexpr int RING = NPH * kBand;
    static_assert(RING >= WS + 1, "the ring must hold a window and the row leaving it");

    // walker start: the first w-1 product rows (row 0's window lacks only its last row); the
    // row before the first window (slot RING - 1) contributes 0
    int vacc[NWV], ring[NWV][RING];
#pragma unroll
    for (int k = 0; k < NWV; ++k) {
        vacc[k] = 0;
#pragma unroll
        for (int j = 0; j < RING; ++j) ring[k][j] = 0;
        const int w = tid + k * kThreads;
        if (w < CW * DC) {
            const int xp = w / DC, dd = w - xp * DC;
            const uint8_t *rc = sref + REFE + xp;
            const uint8_t *tc = stgt + a.tgt_e + xp + (a.Dp - 1) - (d0 + dd);
            int s0 = 0;
#pragma unroll
            for (int i = 0; i < WS - 1; ++i) {
                ring[k][i] = (int)rc[i * RP] * (int)tc[i * TP];
                s0 += ring[k][i];
            }
            vacc[k] = s0;
        }
    }
    // window statistics of a band (global loads, stored to shared memory after the band's
    // vertical pass); each band's loads are issued one band ahead to hide their latency
    auto load_stats = [&](int2 (&st)[NST], int yb) {
        const int nr = min(kBand, QH - yb);
#pragma unroll
        for (int k = 0; k < NST; ++k) {
            const int e = tid + k * kThreads;
            st[k] = make_int2(0, 0);
            if (yb < QH && e < kBand * (QW + TSW)) {
                const int r = e / (QW + TSW), c = e - r * (QW + TSW);
                if (r < nr) {
                    const size_t prow = (size_t)(y0 - RB + yb + r + a.pad_top) * a.pad_w;
                    st[k] = c < QW ? __ldg(a.ref_stats + prow + x0 - RB + a.pad_left + c)
                                   : __ldg(a.tgt_stats + prow + x0 - RB + a.pad_left - d0 - (DC - 1) + (c - QW));
                }
            }
        }
    };
    int2 stv[NST];
    load_stats(stv, 0);
    auto band = [&](auto phase, int yb0) {
        constexpr int PH = decltype(phase)::value;
        if (yb0 >= QH) return;
        const int nrows = min(kBand, QH - yb0);
        int2 stn[NST];
        load_stats(stn, yb0 + kBand);
        // vertical pass, in sub-bands of at most kSub rows: the product rows entering those
        // rows' windows, all loads first, then the running sums (the leaving row read back
        // from the ring) and their stores
        constexpr int kSub = kBand < 6 ? kBand : 6;
        static_assert(kBand % kSub == 0, "a band is a whole number of sub-bands");
        static_for<kBand / kSub>([&](auto sub) {
            constexpr int R0 = decltype(sub)::value * kSub;
            int pn[NWV][kSub];
#pragma unroll
            for (int k = 0; k < NWV; ++k) {
                const int w = tid + k * kThreads;
                const int xp = w / DC, dd = w - xp * DC;
                const bool on = w < CW * DC;
                const uint8_t *rc = sref + REFE + (on ? xp : 0);
                const uint8_t *tc = stgt + a.tgt_e + (on ? xp + (a.Dp - 1) - (d0 + dd) : 0);
#pragma unroll
                for (int r = 0; r < kSub; ++r) {
                    const bool live = on && R0 + r < nrows;
                    const int ya = live ? yb0 + R0 + r + WS - 1 : 0;
                    pn[k][r] = live ? (int)rc[ya * RP] * (int)tc[ya * TP] : 0;
                }
            }
#pragma unroll
            for (int k = 0; k < NWV; ++k) {
                const int w = tid + k * kThreads;
                if (w < CW * DC) {
                    int *vo = vband + w;            // [r][xp][dd] with xp * DC + dd = w
                    int acc = vacc[k];
#pragma unroll
                    for (int r = 0; r < kSub; ++r) {
                        if (R0 + r < nrows) {
                            constexpr int base = PH * kBand + R0;
                            acc += pn[k][r] - ring[k][(base + r + RING - 1) % RING];
                            ring[k][(base + r + WS - 1) % RING] = pn[k][r];
                            vo[(R0 + r) * CW * DC] = acc;
                        }
                    }
                    vacc[k] = acc;
                }
            }
        });
#pragma unroll
        for (int k = 0; k < NST; ++k) {
            const int e = tid + k * kThreads;
            if (e < kBand * (QW + TSW)) {
                const int r = e / (QW + TSW), c = e - r * (QW + TSW);
                if (c < QW) sstr[r * QW + c] = stv[k];
                else sstt[r * TSW + (c - QW)] = stv[k];
            }
        }
        group_sync<BAR, NT>();
        // horizontal pass: item = (band row, disparity quad, column segment).  Neighbouring
        // lanes must read vband's 16-byte units in distinct bank groups: with an odd number of
        // quads (stride kSeg * NQ units between segments, odd) the segment index runs fastest;
        // with an even number it would repeat every two segments, so there the quad runs
        // fastest (units dq + kSeg * NQ * seg: four quads, then the next segment 4 units on)
        const int nitems = nrows * NSEG * NQ;
        for (int it = tid; it < nitems; it += kThreads) {
            int seg, dq, r;
            if constexpr (NQ % 2 == 0) {
                dq = it % NQ;
                const int rs = it / NQ;
                seg = rs % NSEG;
                r = rs / NSEG;
            } else {
                seg = it % NSEG;
                const int rq = it / NSEG;
                dq = rq % NQ;
                r = rq / NQ;
            }
            const int yq = yb0 + r;
            const int xs = seg * kSeg;
            const int nout = min(kSeg, QW - xs);
            const int4 *vr = reinterpret_cast<const int4 *>(vband) + (size_t)r * CW * NQ + dq;
            const int2 *rsr = sstr + r * QW;
            const int2 *tsr = sstt + r * TSW + (DC - 1) - 4 * dq;   // column of x - d for d = d0 + 4dq
            int4 v[kSeg + WS - 1];
            int2 rs[kSeg], ts[kSeg + 3];
#pragma unroll
            for (int j = 0; j < kSeg + WS - 1; ++j)
                v[j] = (j < nout + WS - 1) ? vr[(xs + j) * NQ] : make_int4(0, 0, 0, 0);
#pragma unroll
            for (int j = 0; j < kSeg; ++j) rs[j] = (j < nout) ? rsr[xs + j] : make_int2(0, 0);
#pragma unroll
            for (int j = 0; j < kSeg + 3; ++j) ts[j] = (j < nout + 3) ? tsr[xs + j - 3] : make_int2(0, 0);
            float4 out[kSeg];
            int4 S = make_int4(0, 0, 0, 0);
#pragma unroll
            for (int j = 0; j < WS; ++j) {
                S.x += v[j].x;
                S.y += v[j].y;
                S.z += v[j].z;
                S.w += v[j].w;
            }
#pragma unroll
            for (int j = 0; j < kSeg; ++j) {
                const float ir = __int_as_float(rs[j].y);
                const int2 t0 = ts[j + 3], t1 = ts[j + 2], t2 = ts[j + 1], t3 = ts[j];
                out[j].x = fmaf(-(float)(a.n * S.x - rs[j].x * t0.x), ir * __int_as_float(t0.y), 1.0f);
                out[j].y = fmaf(-(float)(a.n * S.y - rs[j].x * t1.x), ir * __int_as_float(t1.y), 1.0f);
                out[j].z = fmaf(-(float)(a.n * S.z - rs[j].x * t2.x), ir * __int_as_float(t2.y), 1.0f);
                out[j].w = fmaf(-(float)(a.n * S.w - rs[j].x * t3.x), ir * __int_as_float(t3.y), 1.0f);
                if (j + 1 < kSeg) {
                    S.x += v[j + WS].x - v[j].x;
                    S.y += v[j + WS].y - v[j].y;
                    S.z += v[j + WS].z - v[j].z;
                    S.w += v[j + WS].w - v[j].w;
                }
            }
            if constexpr (SWZ) {
                // 16 disparities per position as two 16-byte halves, the half index XORed with
                // bit 2 of the column (the tensor-core aggregation's ldmatrix layout)
                static_assert(DC == 16, "the swizzled layout holds 16 disparities per position");
                T *co = cbuf + (size_t)yq * crow + 4 * (dq & 1);
#pragma unroll
                for (int j = 0; j < kSeg; ++j) {
                    const int x = xs + j;
                    if (j < nout) CostStore<T>::store4(co + (size_t)x * DC + ((((dq >> 1) ^ (x >> 2)) & 1) << 3), out[j]);
                }
            } else {
                T *co = cbuf + (size_t)yq * crow + 4 * dq;
#pragma unroll
                for (int j = 0; j < kSeg; ++j)
                    if (j < nout) CostStore<T>::store4(co + (size_t)(xs + j) * DC, out[j]);
            }
        }
        group_sync<BAR, NT>();
#pragma unroll
        for (int k = 0; k < NST; ++k) stv[k] = stn[k];
    };
    for (int yb0 = 0; yb0 < QH; yb0 += RING)
        static_for<NPH>([&](auto ph) { band(ph, yb0 + decltype(ph)::value * kBand); });
}

// ------------------------------------------------------------- tensor-core cost phase
// mma.sync m16n8k16, FP16 operands, FP32 accumulators: d (4 floats) += A (16 x 16) B (16 x 8).
__device__ __forceinline__ void mma_f16_16816(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1)
{
    asm("mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
        "{%0, %1, %2, %3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// The bytes p[0], p[1] as a packed FP16 pair (p[0] in the low half), exactly: each byte b goes
// into a half whose high byte is 0x64 (the FP16 number 1024 + b), then 1024 is subtracted.
__device__ __forceinline__ uint32_t u8pair_h2(const uint8_t *p)
{
    const uint32_t w = __byte_perm((uint32_t)p[0], (uint32_t)p[1], 0x5410) | 0x64006400u;
    const __half2 h = __hsub2(*reinterpret_cast<const __half2 *>(&w), __half2half2(__ushort_as_half(0x6400)));
    return *reinterpret_cast<const uint32_t *>(&h);
}

template <typename T> __device__ __forceinline__ T cost_from_float(float c);
template <> __device__ __forceinline__ float cost_from_float<float>(float c) { return c; }
template <> __device__ __forceinline__ __half cost_from_float<__half>(float c) { return __float2half_rn(c); }
template <> __device__ __forceinline__ __nv_bfloat16 cost_from_float<__nv_bfloat16>(float c)
{
    return __float2bfloat16_rn(c);
}

// The costs of one chunk of DC <= 16 disparities at the tile plus its bilateral halo (QH x QW
// positions), eq. (c), with the cross term S = sum_block I_ref(q) I_tar(q - d) on the tensor
// cores.  The 8-bit intensities are exact in FP16, every product and every window sum is an
// integer below 2^24, so FP32 accumulation keeps S exact.  One warp owns a block of 8 cost
// columns and walks down its rows; for every staged row the products of that row are one mma
// per 16 product columns:
//   A[m][kk] = I_tar(row, x0b + kk - (d0 + m))   (16 disparities x 16 product columns, Toeplitz)
//   B[kk][n] = I_ref(row, x0b + kk) if 0 <= kk - n <= 2 r_w, else 0   (banded)
// and the accumulator carries S(row window) from row to row: the row entering the window is
// added, the row leaving it is subtracted (B negated).  A row's fragments are built once and
// kept in a register ring of w slots until the row leaves (for w = 11, where two k-steps make
// the ring too large, the leaving row is rebuilt).  Then c = 1 - (n S - S_ref S_tar) r_ref r_tar:
// every lane holds one window-statistics entry per row (lanes 0..7 the reference at the
// block's 8 columns, lanes 8.. the target at x - d), loaded from device memory a window of rows
// ahead, and the formula gathers them with warp shuffles.  Warps work independently; the
// caller synchronises before reading cbuf.  With SWZ the 16 disparities of a position are
// stored as two 16-byte halves swizzled by bit 2 of the column.
template <int RB, int DC, int RW, typename T, int TX, int TY, int NT = kThreads, bool SWZ = false>
__device__ __forceinline__ void cost_chunk_mma(const FusedArgs &a, const uint8_t *sref, const uint8_t *stgt,
                                               T *cbuf, int x0, int y0, int d0, int tid)
{
    static_assert(DC <= 16, "one block of 16 disparities per mma");
    static_assert(!SWZ || DC == 16, "the swizzled layout holds 16 disparities per position");
    constexpr int QH = TY + 2 * RB, QW = TX + 2 * RB;
    constexpr int NR = 2 * RW + 1;                     // rows of a window
    constexpr int NXB = (QW + 7) / 8;                  // column blocks (one warp each at a time)
    constexpr int NKC = (8 + 2 * RW + 15) / 16;        // k-steps per row: 8 + 2 r_w product columns
    constexpr bool RING = NKC == 1;                    // keep every row's fragments until it leaves
    constexpr int MM = RW + RB;
    constexpr int REFE = (MM + 15) / 16 * 16 - MM;
    constexpr int RP = (REFE + TX + 2 * MM + 15) / 16 * 16;
    const int TP = a.tgt_box_w;
    const int warp = tid >> 5, lane = tid & 31, g = lane >> 2, t4 = lane & 3;
    const size_t crow = (size_t)QW * DC;
    // B masks per k-step: K slot kk is in the window of output column g iff 0 <= kk - g <= 2 r_w
    uint32_t mlo[NKC], mhi[NKC];
#pragma unroll
    for (int kc = 0; kc < NKC; ++kc) {
        auto hm = [&](int kk) { return (kk - g >= 0 && kk - g <= 2 * RW) ? 0xffffu : 0u; };
        const int k0 = 16 * kc + 2 * t4;
        mlo[kc] = hm(k0) | (hm(k0 + 1) << 16);
        mhi[kc] = hm(k0 + 8) | (hm(k0 + 9) << 16);
    }
    // shuffle sources of this lane's four outputs (x = xa + (k & 1), d = d0 + g + 8 (k >> 1)):
    // the reference entry of x, the target entry of x - d
    int src_r[2], src_t[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int xr = 2 * t4 + (k & 1), dd = g + (k >> 1) * 8;
        if (k < 2) src_r[k] = xr;
        src_t[k] = min(max(8 + xr - dd + DC - 1, 0), 31);
    }
    for (int xb = warp; xb < NXB; xb += NT / 32) {
        const int x0b = xb * 8;
        const uint8_t *rb = sref + REFE + x0b + 2 * t4;
        const uint8_t *tb = stgt + a.tgt_e + (a.Dp - 1) - d0 + x0b + 2 * t4 - g;
        // this lane's statistics entry at row 0; columns past the tile are clamped (their costs
        // are not stored)
        const int2 *esrc = nullptr;
        {
            const size_t prow0 = (size_t)(y0 - RB + a.pad_top) * a.pad_w + x0 - RB + a.pad_left;
            if (lane < 8) esrc = a.ref_stats + prow0 + min(x0b + lane, QW - 1);
            else if (lane < DC + 15) esrc = a.tgt_stats + prow0 + min(x0b - d0 - DC + 1 + (lane - 8), QW - 1 - d0);
        }
        auto ld_stats = [&](int yq) { return (esrc && yq < QH) ? __ldg(esrc + (size_t)yq * a.pad_w) : make_int2(0, 0); };

        // fragments of one staged row: a0 = A[g][2t4 + {0,1}], a1 = A[g + 8][...], a2 =
        // A[g][2t4 + 8 + {0,1}] (a3 = A[g + 8][2t4 + 8 + {0,1}] = a0, Toeplitz); b0 = B[2t4 +
        // {0,1}][g], b1 = B[2t4 + 8 + {0,1}][g]
        auto build = [&](int row, uint32_t (&f)[NKC][5]) {
            const uint8_t *rr = rb + row * RP;
            const uint8_t *tr = tb + row * TP;
#pragma unroll
            for (int kc = 0; kc < NKC; ++kc) {
                f[kc][0] = u8pair_h2(tr + 16 * kc);
                f[kc][1] = u8pair_h2(tr + 16 * kc - 8);
                f[kc][2] = u8pair_h2(tr + 16 * kc + 8);
                f[kc][3] = u8pair_h2(rr + 16 * kc) & mlo[kc];
                f[kc][4] = u8pair_h2(rr + 16 * kc + 8) & mhi[kc];
            }
        };
        float acc[4] = {0.f, 0.f, 0.f, 0.f};
        auto apply = [&](const uint32_t (&f)[NKC][5], uint32_t sign) {   // sign 0x80008000 negates B
#pragma unroll
            for (int kc = 0; kc < NKC; ++kc) {
                const uint32_t af[4] = {f[kc][0], f[kc][1], f[kc][2], f[kc][0]};
                mma_f16_16816(acc, af, f[kc][3] ^ sign, f[kc][4] ^ sign);
            }
        };
        // c of this lane's four outputs at cost row yq from S = acc and the row's entries e
        auto emit = [&](int yq, int2 e) {
            const int xa = x0b + 2 * t4;
            int2 rs[2], ts[4];
#pragma unroll
            for (int k = 0; k < 2; ++k)
                rs[k] = make_int2(__shfl_sync(0xffffffffu, e.x, src_r[k]), __shfl_sync(0xffffffffu, e.y, src_r[k]));
#pragma unroll
            for (int k = 0; k < 4; ++k)
                ts[k] = make_int2(__shfl_sync(0xffffffffu, e.x, src_t[k]), __shfl_sync(0xffffffffu, e.y, src_t[k]));
            T *co = cbuf + (size_t)yq * crow;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int x = xa + (k & 1), dd = g + (k >> 1) * 8;
                if (x < QW && dd < DC) {
                    const int S = __float_as_int(acc[k] + 8388608.f) - 0x4B000000;   // exact, 0 <= S < 2^23
                    const int2 r = rs[k & 1], t = ts[k];
                    const float c = fmaf(-(float)(a.n * S - r.x * t.x), __int_as_float(r.y) * __int_as_float(t.y), 1.0f);
                    size_t o = (size_t)x * DC + dd;
                    if constexpr (SWZ) o = (size_t)x * DC + ((((dd >> 3) ^ (x >> 2)) & 1) << 3) + (dd & 7);
                    co[o] = cost_from_float<T>(c);
                }
            }
        };

        int2 scur[NR], snxt[NR];
#pragma unroll
        for (int j = 0; j < NR; ++j) scur[j] = ld_stats(j);
        if constexpr (RING) {
            // row r lives in slot r % NR from the step it enters (r - 2 r_w) to the step it leaves (r)
            uint32_t fr[NR][NKC][5];
#pragma unroll
            for (int i = 0; i < NR - 1; ++i) {
                build(i, fr[i]);
                apply(fr[i], 0u);
            }
            for (int yq0 = 0; yq0 < QH; yq0 += NR) {
#pragma unroll
                for (int j = 0; j < NR; ++j) snxt[j] = ld_stats(yq0 + NR + j);
#pragma unroll
                for (int j = 0; j < NR; ++j) {
                    const int yq = yq0 + j;
                    if (yq < QH) {
                        build(yq + 2 * RW, fr[(j + 2 * RW) % NR]);
                        apply(fr[(j + 2 * RW) % NR], 0u);
                        emit(yq, scur[j]);
                        apply(fr[j], 0x80008000u);   // the leaving row yq (slot yq % NR = j)
                    }
                }
#pragma unroll
                for (int j = 0; j < NR; ++j) scur[j] = snxt[j];
            }
        } else {
            uint32_t fn[NKC][5], fo[NKC][5];
            for (int i = 0; i < NR - 1; ++i) {
                build(i, fn);
                apply(fn, 0u);
            }
            for (int yq0 = 0; yq0 < QH; yq0 += NR) {
#pragma unroll
                for (int j = 0; j < NR; ++j) snxt[j] = ld_stats(yq0 + NR + j);
#pragma unroll
                for (int j = 0; j < NR; ++j) {
                    const int yq = yq0 + j;
                    if (yq < QH) {
                        build(yq + 2 * RW, fn);
                        apply(fn, 0u);
                        emit(yq, scur[j]);
                        build(yq, fo);
                        apply(fo, 0x80008000u);
                    }
                }
#pragma unroll
                for (int j = 0; j < NR; ++j) scur[j] = snxt[j];
            }
        }
    }
}

// B2: also track the smallest E over d != d* and write best2 (a separate instantiation, so
// that the kernels without the optional output carry none of its registers or operations).
template <int RB, int DC, typename T, int WC, bool B2 = false>
__global__ void __launch_bounds__(kThreads, 1)
k_fused(const __grid_constant__ PairDesc single, const PairDesc *__restrict__ pairs,
        const int2 *__restrict__ items, int nitems, int *__restrict__ counter)
{
    static_assert(DC % 4 == 0, "DC must be a multiple of 4");
    constexpr int TX = tile_x(WC), TY = tile_y(WC);
    constexpr int KB = 2 * RB + 1;
    constexpr int QH = TY + 2 * RB, QW = TX + 2 * RB;
    constexpr int NR = kPY + 2 * RB;   // neighbour rows seen by one thread's pixel column
    constexpr int NQ = DC / 4;         // disparity quads per chunk
    extern __shared__ __align__(128) uint8_t smem[];
    __shared__ __align__(16) FusedArgs s_args;
    __shared__ int s_item;
    // the mbarrier and the wait flag live at fixed addresses: the dynamic layout moves with
    // each tile's pair (its search range sets the width of the target strip)
    __shared__ __align__(8) uint64_t s_bar;
    __shared__ int s_flag;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const FusedArgs &a = s_args;
    uint64_t *bar = &s_bar;
    int *flag = &s_flag;
    if (tid == 0) mbar_init(bar, 1);

    for (int iter = 0;; ++iter) {
        int tx = 0, ty = 0;
        const PairDesc *pd = claim_tile<kThreads>(single, pairs, items, nitems, counter, iter, s_args, s_item, tid, tx, ty);
        if (!pd) return;

        const int RP = a.ref_box_w, TP = a.tgt_box_w;
        const SmemLayout L = smem_layout(RB, a.m, DC, RP, TP, a.box_h, (int)sizeof(T), TX, TY, 1, 0);
        uint8_t *sref = smem + L.sref;
        uint8_t *stgt = smem + L.stgt;
        T *cbuf = reinterpret_cast<T *>(smem + L.cbuf);
        float *sI = reinterpret_cast<float *>(smem + L.sI);
        float *sK = reinterpret_cast<float *>(smem + L.sK);
        const int x0 = tx * TX, y0 = ty * TY;

        // ---- 1. stage the image tiles with TMA
        for (int i = tid; i < KB * KB; i += kThreads) sK[i] = a.K[i];
        __syncthreads();
        if (!stage_images(pd, a, sref, stgt, bar, flag, x0, y0, iter, tid)) return;

    const int rw = a.rw;
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

    const int xt = (warp % WC) * 32 + lane;
    const int yt0 = (warp / WC) * kPY;
    float Ip[kPY];
#pragma unroll
    for (int i = 0; i < kPY; ++i) Ip[i] = sI[(yt0 + i + RB) * QW + xt + RB];

    float best[kPY], bm1[kPY], bp1[kPY], prev[kPY], sec[B2 ? kPY : 1];
    int bd[kPY];
#pragma unroll
    for (int i = 0; i < kPY; ++i) {
        best[i] = __int_as_float(0x7f800000);
        bm1[i] = bp1[i] = prev[i] = best[i];
        if constexpr (B2) sec[i] = best[i];
        bd[i] = -1;
    }

    const size_t crow = (size_t)QW * DC;   // floats per cost row
    for (int d0 = 0; d0 < a.D; d0 += DC) {
        // ---- 2a/2b. costs of the chunk (block radius dispatched to a compile-time value)
        switch (rw) {
        case 1: cost_chunk_mma<RB, DC, 1, T, TX, TY>(a, sref, stgt, cbuf, x0, y0, d0, tid); break;
        case 2: cost_chunk_mma<RB, DC, 2, T, TX, TY>(a, sref, stgt, cbuf, x0, y0, d0, tid); break;
        case 3: cost_chunk_mma<RB, DC, 3, T, TX, TY>(a, sref, stgt, cbuf, x0, y0, d0, tid); break;
        case 4: cost_chunk_mma<RB, DC, 4, T, TX, TY>(a, sref, stgt, cbuf, x0, y0, d0, tid); break;
        default: cost_chunk_mma<RB, DC, 5, T, TX, TY>(a, sref, stgt, cbuf, x0, y0, d0, tid); break;
        }
        __syncthreads();
        // ---- 2c. bilateral aggregation of the chunk: each thread kPY pixels x DC d
        float2 acc[kPY][DC / 2];
#pragma unroll
        for (int i = 0; i < kPY; ++i)
#pragma unroll
            for (int k = 0; k < DC / 2; ++k) acc[i][k] = make_float2(0.f, 0.f);
        for (int dx = 0; dx < KB; ++dx) {
            float Kr[KB];
#pragma unroll
            for (int j = 0; j < KB; ++j) Kr[j] = sK[dx * KB + j];
            const T *cb = cbuf + ((size_t)yt0 * QW + xt + dx) * DC;
            const float *ib = sI + yt0 * QW + xt + dx;
            // software pipeline over neighbour rows: while row r is accumulated, the
            // costs of row r+1 are in flight and its weights are being computed
            float2 q[2 * NQ];
#pragma unroll
            for (int k = 0; k < NQ; ++k) CostStore<T>::load4(cb + 4 * k, q[2 * k], q[2 * k + 1]);
            float wgt[kPY];
            {
                const float Iq = ib[0];
#pragma unroll
                for (int i = 0; i < kPY; ++i) {
                    const int dy = 0 - i;
                    if (dy >= 0 && dy <= 2 * RB) {
                        const float t = Iq - Ip[i];
                        wgt[i] = ex2_approx(fmaf(-t, t, Kr[dy]));
                    }
                }
            }
#pragma unroll
            for (int r = 0; r < NR; ++r) {
                float2 qn[2 * NQ];
                float wn[kPY];
                if (r + 1 < NR) {
#pragma unroll
                    for (int k = 0; k < NQ; ++k)
                        CostStore<T>::load4(cb + (r + 1) * crow + 4 * k, qn[2 * k], qn[2 * k + 1]);
                    const float Iq = ib[(r + 1) * QW];
#pragma unroll
                    for (int i = 0; i < kPY; ++i) {
                        const int dy = r + 1 - i;      // neighbour row - pixel row + RB
                        if (dy >= 0 && dy <= 2 * RB) {
                            const float t = Iq - Ip[i];
                            wn[i] = ex2_approx(fmaf(-t, t, Kr[dy]));
                        }
                    }
                }
#pragma unroll
                for (int i = 0; i < kPY; ++i) {
                    const int dy = r - i;
                    if (dy >= 0 && dy <= 2 * RB) {
                        const float2 w2 = make_float2(wgt[i], wgt[i]);
#pragma unroll
                        for (int k = 0; k < 2 * NQ; ++k) acc[i][k] = __ffma2_rn(w2, q[k], acc[i][k]);
                    }
                }
                if (r + 1 < NR) {
#pragma unroll
                    for (int k = 0; k < 2 * NQ; ++k) q[k] = qn[k];
#pragma unroll
                    for (int i = 0; i < kPY; ++i) wgt[i] = wn[i];
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
                    if constexpr (B2) sec[i] = best[i];
                    best[i] = v;
                    bd[i] = d;
                    bm1[i] = prev[i];
                } else {
                    if constexpr (B2) sec[i] = fminf(sec[i], v);
                    if (d == bd[i] + 1) bp1[i] = v;
                }
                prev[i] = v;
            }
        __syncthreads();
    }

    // ---- 3. epilogue: eq. (subpixel), add back s_i(v), validity from the row table
#pragma unroll
    for (int i = 0; i < kPY; ++i) {
        const int u = x0 + xt, v = y0 + yt0 + i;
        if (u >= a.W || v >= a.H) continue;
        const int4 rt = __ldg(a.row_tab + v);   // {s_i(v), max s_i, min s_i over v +- m}
        float delta = 0.f;
        if (bd[i] > 0 && bd[i] < a.D - 1) {
            const float den = 2.f * bm1[i] + 2.f * bp1[i] - 4.f * best[i];
            if (den > 0.f) delta = (bm1[i] - bp1[i]) / den;
        }
        const size_t o = (size_t)v * a.W + u;
        a.disp[o] = (float)bd[i] + delta + (float)rt.x;
        if (a.wta) a.wta[o] = bd[i];
        if (a.valid) {
            const int ulo = a.m + a.D - 1 + max(0, rt.y);
            const int uhi = a.W - 1 - a.m + min(0, rt.z);
            a.valid[o] = (uint8_t)(v >= a.m && v <= a.H - 1 - a.m && u >= ulo && u <= uhi);
        }
        if constexpr (B2) {
            // the skipped normaliser sum_q w(p,q) (out-of-image q carry weight 0)
            float ws = 0.f;
            for (int dx = 0; dx < KB; ++dx)
                for (int dy = 0; dy < KB; ++dy) {
                    const float t = sI[(yt0 + i + dy) * QW + xt + dx] - Ip[i];
                    ws += ex2_approx(fmaf(-t, t, sK[dx * KB + dy]));
                }
            a.best2[2 * o] = best[i] / ws;
            a.best2[2 * o + 1] = sec[i] / ws;
        }
    }
    }  // tile loop
}

// Named barriers of the warp-specialised kernel (0 is __syncthreads).
enum { kBarFull0 = 1, kBarFull1 = 2, kBarEmpty0 = 3, kBarEmpty1 = 4, kBarProd = 5 };

__device__ __forceinline__ void named_sync(int id, int n)
{
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory");
}

__device__ __forceinline__ void named_arrive(int id, int n)
{
    asm volatile("bar.arrive %0, %1;" ::"r"(id), "r"(n) : "memory");
}

// The fused kernel with its two phases on separate warps.  Producer warps (kWsProdWarps)
// compute the costs of chunk k+1 (eq. c, the same integer passes as cost_chunk) into one of
// two cost buffers while the consumer warps (kWsConsWarps) aggregate chunk k from the other
// (eq. fbs) and keep the running WTA; "full" and "empty" named barriers hand each buffer
// over.  Tiles are 64 x 16; the persistent tile loop, the staging and the epilogue are those
// of k_fused.
template <int RB, int DC, typename T>
__global__ void __launch_bounds__(kWsThreads, 1)
k_fused_ws(const __grid_constant__ PairDesc single, const PairDesc *__restrict__ pairs,
           const int2 *__restrict__ items, int nitems, int *__restrict__ counter)
{
    static_assert(DC % 4 == 0, "DC must be a multiple of 4");
    constexpr int TX = tile_x(kWsWC), TY = tile_y(kWsWC);
    constexpr int KB = 2 * RB + 1;
    constexpr int QH = TY + 2 * RB, QW = TX + 2 * RB;
    constexpr int NR = kWsPY + 2 * RB;
    constexpr int NQ = DC / 4;
    constexpr int NPT = 32 * kWsProdWarps;      // producer threads
    extern __shared__ __align__(128) uint8_t smem[];
    __shared__ __align__(16) FusedArgs s_args;
    __shared__ int s_item;
    __shared__ __align__(8) uint64_t s_bar;
    __shared__ int s_flag;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const FusedArgs &a = s_args;
    uint64_t *bar = &s_bar;
    int *flag = &s_flag;
    if (tid == 0) mbar_init(bar, 1);

    for (int iter = 0;; ++iter) {
        int tx = 0, ty = 0;
        const PairDesc *pd = claim_tile<kWsThreads>(single, pairs, items, nitems, counter, iter, s_args, s_item, tid, tx, ty);
        if (!pd) return;

        const int RP = a.ref_box_w, TP = a.tgt_box_w;
        const SmemLayout L = smem_layout(RB, a.m, DC, RP, TP, a.box_h, (int)sizeof(T), TX, TY, 2, kWsBand);
        uint8_t *sref = smem + L.sref;
        uint8_t *stgt = smem + L.stgt;
        T *cbuf0 = reinterpret_cast<T *>(smem + L.cbuf);
        T *cbuf1 = reinterpret_cast<T *>(smem + L.cbuf1);
        int *vband = reinterpret_cast<int *>(smem + L.vband);
        int2 *sstr = reinterpret_cast<int2 *>(smem + L.sstr);
        int2 *sstt = reinterpret_cast<int2 *>(smem + L.sstt);
        float *sI = reinterpret_cast<float *>(smem + L.sI);
        float *sK = reinterpret_cast<float *>(smem + L.sK);
        const int x0 = tx * TX, y0 = ty * TY;

        // ---- 1. stage the image tiles with TMA
        for (int i = tid; i < KB * KB; i += kWsThreads) sK[i] = a.K[i];
        __syncthreads();
        if (!stage_images(pd, a, sref, stgt, bar, flag, x0, y0, iter, tid)) return;

        const int rw = a.rw;
        for (int i = tid; i < QH * QW; i += kWsThreads) {
            const int yq = i / QW, xq = i - yq * QW;
            const int ix = x0 - RB + xq, iy = y0 - RB + yq;
            float v = 1e18f;
            if (ix >= 0 && ix < a.W && iy >= 0 && iy < a.H)
                v = (float)sref[(yq + rw) * RP + a.ref_e + xq + rw] * a.iscale;
            sI[i] = v;
        }
        __syncthreads();

        const int nchunk = (a.D + DC - 1) / DC;
        if (warp < kWsProdWarps) {
            // ---- producers: costs of chunk k into buffer k & 1, once the consumers are done
            // with what that buffer held (chunk k - 2)
            for (int k = 0; k < nchunk; ++k) {
                const int b = k & 1;
                if (k >= 2) named_sync(b ? kBarEmpty1 : kBarEmpty0, kWsThreads);
                T *cb = b ? cbuf1 : cbuf0;
                switch (rw) {
                case 1: cost_chunk<RB, DC, 1, T, TX, TY, NPT, kBarProd, kWsBand>(a, sref, stgt, cb, vband, sstr, sstt, x0, y0, k * DC, tid); break;
                case 2: cost_chunk<RB, DC, 2, T, TX, TY, NPT, kBarProd, kWsBand>(a, sref, stgt, cb, vband, sstr, sstt, x0, y0, k * DC, tid); break;
                case 3: cost_chunk<RB, DC, 3, T, TX, TY, NPT, kBarProd, kWsBand>(a, sref, stgt, cb, vband, sstr, sstt, x0, y0, k * DC, tid); break;
                case 4: cost_chunk<RB, DC, 4, T, TX, TY, NPT, kBarProd, kWsBand>(a, sref, stgt, cb, vband, sstr, sstt, x0, y0, k * DC, tid); break;
                default: cost_chunk<RB, DC, 5, T, TX, TY, NPT, kBarProd, kWsBand>(a, sref, stgt, cb, vband, sstr, sstt, x0, y0, k * DC, tid); break;
                }
                __threadfence_block();
                named_arrive(b ? kBarFull1 : kBarFull0, kWsThreads);
            }
            // match the consumers' "empty" arrivals of the last two chunks
            for (int k = nchunk < 2 ? 0 : nchunk - 2; k < nchunk; ++k)
                named_sync((k & 1) ? kBarEmpty1 : kBarEmpty0, kWsThreads);
        } else {
            // ---- consumers: aggregation of chunk k, running WTA, then release the buffer
            const int cw = warp - kWsProdWarps;
            const int xt = (cw & 1) * 32 + lane;
            const int yt0 = (cw >> 1) * kWsPY;
            float Ip[kWsPY];
#pragma unroll
            for (int i = 0; i < kWsPY; ++i) Ip[i] = sI[(yt0 + i + RB) * QW + xt + RB];
            float best[kWsPY], bm1[kWsPY], bp1[kWsPY], prev[kWsPY];
            int bd[kWsPY];
#pragma unroll
            for (int i = 0; i < kWsPY; ++i) {
                best[i] = __int_as_float(0x7f800000);
                bm1[i] = bp1[i] = prev[i] = best[i];
                bd[i] = -1;
            }
            const size_t crow = (size_t)QW * DC;
            for (int k = 0; k < nchunk; ++k) {
                const int b = k & 1;
                const int d0 = k * DC;
                named_sync(b ? kBarFull1 : kBarFull0, kWsThreads);
                const T *cbuf = b ? cbuf1 : cbuf0;
                float2 acc[kWsPY][DC / 2];
#pragma unroll
                for (int i = 0; i < kWsPY; ++i)
#pragma unroll
                    for (int q = 0; q < DC / 2; ++q) acc[i][q] = make_float2(0.f, 0.f);
                for (int dx = 0; dx < KB; ++dx) {
                    float Kr[KB];
#pragma unroll
                    for (int j = 0; j < KB; ++j) Kr[j] = sK[dx * KB + j];
                    const T *cb = cbuf + ((size_t)yt0 * QW + xt + dx) * DC;
                    const float *ib = sI + yt0 * QW + xt + dx;
                    float2 q[2 * NQ];
#pragma unroll
                    for (int j = 0; j < NQ; ++j) CostStore<T>::load4(cb + 4 * j, q[2 * j], q[2 * j + 1]);
                    float wgt[kWsPY];
                    {
                        const float Iq = ib[0];
#pragma unroll
                        for (int i = 0; i < kWsPY; ++i) {
                            const int dy = 0 - i;
                            if (dy >= 0 && dy <= 2 * RB) {
                                const float t = Iq - Ip[i];
                                wgt[i] = ex2_approx(fmaf(-t, t, Kr[dy]));
                            }
                        }
                    }
#pragma unroll
                    for (int r = 0; r < NR; ++r) {
                        float2 qn[2 * NQ];
                        float wn[kWsPY];
                        if (r + 1 < NR) {
#pragma unroll
                            for (int j = 0; j < NQ; ++j)
                                CostStore<T>::load4(cb + (r + 1) * crow + 4 * j, qn[2 * j], qn[2 * j + 1]);
                            const float Iq = ib[(r + 1) * QW];
#pragma unroll
                            for (int i = 0; i < kWsPY; ++i) {
                                const int dy = r + 1 - i;
                                if (dy >= 0 && dy <= 2 * RB) {
                                    const float t = Iq - Ip[i];
                                    wn[i] = ex2_approx(fmaf(-t, t, Kr[dy]));
                                }
                            }
                        }
#pragma unroll
                        for (int i = 0; i < kWsPY; ++i) {
                            const int dy = r - i;
                            if (dy >= 0 && dy <= 2 * RB) {
                                const float2 w2 = make_float2(wgt[i], wgt[i]);
#pragma unroll
                                for (int j = 0; j < 2 * NQ; ++j) acc[i][j] = __ffma2_rn(w2, q[j], acc[i][j]);
                            }
                        }
                        if (r + 1 < NR) {
#pragma unroll
                            for (int j = 0; j < 2 * NQ; ++j) q[j] = qn[j];
#pragma unroll
                            for (int i = 0; i < kWsPY; ++i) wgt[i] = wn[i];
                        }
                    }
                }
                // the buffer is free once every consumer has read it
                named_arrive(b ? kBarEmpty1 : kBarEmpty0, kWsThreads);
#pragma unroll
                for (int i = 0; i < kWsPY; ++i)
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
            }
            // ---- epilogue: eq. (subpixel), add back s_i(v), validity from the row table
#pragma unroll
            for (int i = 0; i < kWsPY; ++i) {
                const int u = x0 + xt, v = y0 + yt0 + i;
                if (u >= a.W || v >= a.H) continue;
                const int4 rt = __ldg(a.row_tab + v);
                float delta = 0.f;
                if (bd[i] > 0 && bd[i] < a.D - 1) {
                    const float den = 2.f * bm1[i] + 2.f * bp1[i] - 4.f * best[i];
                    if (den > 0.f) delta = (bm1[i] - bp1[i]) / den;
                }
                const size_t o = (size_t)v * a.W + u;
                a.disp[o] = (float)bd[i] + delta + (float)rt.x;
                if (a.wta) a.wta[o] = bd[i];
                if (a.valid) {
                    const int ulo = a.m + a.D - 1 + max(0, rt.y);
                    const int uhi = a.W - 1 - a.m + min(0, rt.z);
                    a.valid[o] = (uint8_t)(v >= a.m && v <= a.H - 1 - a.m && u >= ulo && u <= uhi);
                }
            }
        }
        // every warp leaves the tile together: the next tile's copies overwrite the buffers
        __syncthreads();
    }
}

typedef void (*FusedKernel)(const PairDesc, const PairDesc *, const int2 *, int, int *);

template <int DC, typename T, int WC, bool B2 = false>
FusedKernel pick_rb(int rb)
{
    switch (rb) {
    case 0: return k_fused<0, DC, T, WC, B2>;
    case 1: return k_fused<1, DC, T, WC, B2>;
    case 2: return k_fused<2, DC, T, WC, B2>;
    case 3: return k_fused<3, DC, T, WC, B2>;
    case 4: return k_fused<4, DC, T, WC, B2>;
    case 5: return k_fused<5, DC, T, WC, B2>;
    case 6: return k_fused<6, DC, T, WC, B2>;
    case 7: return k_fused<7, DC, T, WC, B2>;
    }
    return nullptr;
}

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
