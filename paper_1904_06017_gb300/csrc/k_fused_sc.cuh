// k_fused_sc.cuh -- the FP32 fused step (eq. c, eq. omega_s, eq. fbs, WTA, eq. subpixel, §3.2)
// with certified tensor-core screening: its outputs are bit for bit those of k_fused, the plain
// FP32 kernel, at a fraction of the FP32 arithmetic.
//
// Screening.  Per chunk of 32 disparities the costs c32 of the tile plus its bilateral halo are
// computed in FP32 (cost_chunk, exact integer numerators) and stored as c16 = RN16(2^8 c32); the
// aggregation E(p, d) = sum_q w(p, q) c(q, d) runs on the tensor cores (mma.sync m16n8k16, FP16
// operands, FP32 accumulators) over 4 x 4 pixel patches, with the weights w16 = RN16(2^12 w32)
// formed in FP32 from k_fused's own exponent.  Every weight and cost is non-negative and each is
// rounded once to FP16 (relative error 2^-11 in the normal range), so for every (p, d)
//     |E16 - 2^20 E32| <= eps 2^20 E32 + a,
// where E32 is k_fused's FP32 sum: eps covers the two FP16 roundings of each product (2^-10),
// the tensor core's FP32 accumulation (at most 17 terms per k-step, 14 k-steps, each addition
// within 2^-23 of the running sum, truncating or rounding: 2.8e-5), k_fused's own chain of 121
// FMAs (7.2e-6) and the ex2 / exponent roundings of the scaled weight (1e-5): 1.02e-3, taken as
// 1.1e-3; a (64, i.e. 6.1e-5 unscaled) covers FP16 subnormal weights and costs even if the
// tensor core flushed them.  Hence the FP32 argmin d* (lowest d on ties) satisfies
//     E16(d*) <= thr(min_d E16) = (min_d E16 + a) (1 + eps) / (1 - eps) + a,
// and so does every d that ties it.  Each pixel keeps the range [dlo, dhi] that holds every d
// with E16(d) <= thr(running minimum); a chunk whose minimum m makes thr(m) smaller than the
// previous minimum drops the earlier range (none of its disparities can satisfy the final test).
//
// Refinement.  After the last chunk the tile refines [dlo - 1, dhi + 1] of every pixel with
// k_fused's arithmetic: FP32 costs from the tensor-core cost phase (cost_chunk_mma, bit for bit
// k_fused's), the weight ex2(fma(-t, t, K)), and the 121-term FMA chain in k_fused's order
// (window column outer, row inner), then k_fused's running WTA in increasing d.  The winner and
// its two neighbours (the parabola of eq. subpixel) are therefore k_fused's values exactly.
// With the best2 output (B2) every pixel refines all D disparities (a diagnostic path).
#pragma once
#include "k_fused_tc.cuh"

namespace sgb {

constexpr int kScDC = 32;       // disparities per screening chunk
constexpr int kScDCR = 8;       // disparities per FP32 refinement chunk
constexpr int kScBand = 6;      // cost rows per band of the screening chunk's cost phase
constexpr int kScQWI = 44;      // row length of the staged FP32 intensities (>= QW, >= 28 + 16)
// Refinement planes: rows of kScRPW entries (8 mod 32) and planes a multiple of 32 entries
// apart, so that the warp's 8 x 4 pixels read 32 distinct banks whatever disparity each needs
constexpr int kScRPW = 72;
__host__ __device__ constexpr int sc_psz(int qh) { return (qh * kScRPW + 31) / 32 * 32; }
constexpr int kScWSh = 12;      // weights scaled by 2^12 before rounding to FP16
constexpr int kScCSh = 8;       // costs scaled by 2^8
constexpr float kScEps = 1.1e-3f;
constexpr float kScAbs = 64.f;  // in the scaled units of E16 (2^20 x E32)
// (1 + eps) / (1 - eps), rounded up
constexpr float kScRho = (1.0f + kScEps) / (1.0f - kScEps) + 1e-6f;

constexpr int kScRefOff = 16384;   // bytes into escr: past the refinement's window sums (<= 10 KB)

__device__ __forceinline__ float sc_thr(float m) { return fmaf(m + kScAbs, kScRho, kScAbs); }

// Shared memory of the screened form (offsets from the 128-byte aligned dynamic base):
//   sref, stgt  image tiles (TMA), as in k_fused
//   cbuf   screening: [QH][QW][32] FP16 costs (16-byte units swizzled by bits 1..2 of the
//          column); refinement: 8 FP32 planes of [QH][kScRPW], sc_psz(QH) entries apart -- the
//          same bytes
//   escr   the cost phase's vertical window sums ([band][CW][32] i32); the same bytes hold the
//          per-warp E blocks of the aggregation ([warp][2][16 pixels][32] f32, 16-byte units
//          swizzled by the pixel); during the refinement, from kScRefOff on: the intensities
//          again as [QH][kScRPW] f32, and the spatial exponents as [2 RB + 1][12] f32
//   sstr, sstt  window statistics of one band
//   sI     [QH][kScQWI] f32  the reference intensities times sqrt(log2 e) / sigma1 of the cost
//          positions (1e18 outside the image, as in k_fused)
//   skxy   [4 + 2 RB][32][8] f32  -(K[dx][dy] + 12) of this lane's eight A-fragment weights per
//          window row (1e30 outside the window)
struct ScLayout {
    size_t sref, stgt, cbuf, escr, sstr, sstt, sI, skxy, total;
};

__host__ __device__ inline ScLayout sc_layout(int rb, int m, int ref_box_w, int tgt_box_w, int box_h)
{
    ScLayout L;
    const int TX = tile_x(kScWC), TY = tile_y(kScWC);
    const int QH = TY + 2 * rb, QW = TX + 2 * rb, CW = TX + 2 * m, NKS = 4 + 2 * rb;
    const size_t vb = (size_t)kScBand * CW * kScDC * 4, eb = (size_t)kWarps * 2 * 16 * kScDC * 4;
    const size_t c16 = (size_t)QH * QW * kScDC * 2, c32 = (size_t)kScDCR * sc_psz(QH) * 4;
    L.sref = 0;
    L.stgt = align_up((size_t)box_h * ref_box_w, 128);
    L.cbuf = align_up(L.stgt + (size_t)box_h * tgt_box_w, 128);
    L.escr = align_up(L.cbuf + (c16 > c32 ? c16 : c32), 128);
    L.sstr = align_up(L.escr + (vb > eb ? vb : eb), 16);
    L.sstt = align_up(L.sstr + (size_t)kScBand * QW * 8, 16);
    L.sI = align_up(L.sstt + (size_t)kScBand * (QW + kScDC - 1) * 8, 16);
    L.skxy = align_up(L.sI + (size_t)QH * kScQWI * 4, 16);
    L.total = align_up(L.skxy + (size_t)NKS * 32 * 32, 128);
    return L;
}

// Two FP32 values as a packed FP16 pair (lo in the low half), each rounded to nearest.
__device__ __forceinline__ uint32_t h2_rn(float lo, float hi)
{
    uint32_t r;
    asm("cvt.rn.f16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
    return r;
}

// The E blocks of the per-warp scratch: pixel row m of a patch holds 32 floats as eight
// 16-byte units, unit u stored at u ^ (m & 7) (conflict-free fragment stores and row reads).
__device__ __forceinline__ int sc_eunit(int u, int m) { return u ^ (m & 7); }

template <int RB, bool B2 = false>
__global__ void __launch_bounds__(kThreads, 1)
k_fused_sc(const __grid_constant__ PairDesc single, const PairDesc *__restrict__ pairs,
           const int2 *__restrict__ items, int nitems, int *__restrict__ counter)
{
    using X = TcOps<__half>;
    constexpr int DC = kScDC, DCR = kScDCR;
    constexpr int TX = tile_x(kScWC), TY = tile_y(kScWC);
    constexpr int KB = 2 * RB + 1;
    constexpr int QH = TY + 2 * RB, QW = TX + 2 * RB;
    constexpr int QWI = kScQWI;
    constexpr int NKS = 4 + 2 * RB;              // k-steps: the window rows of a patch
    constexpr int NPX = TX / 4, NPY = TY / 4;    // patches of the tile
    constexpr int NPW = NPX * NPY / kWarps;      // patches per warp
    constexpr int NPP = NPW / 2;                 // handled two at a time; also pixels per lane
    static_assert(RB <= kScMaxRB && NKS <= 16 && QW + 2 <= QWI, "a window row spans at most 16 columns");
    static_assert((NPX * NPY) % kWarps == 0 && NPW % 2 == 0, "patches must split evenly over the warps");
    static_assert(kScBand * (TX + 2 * (RB + kMaxRW)) * kScDCR * 4 <= kScRefOff, "refinement window sums");
    static_assert(kScRefOff + (QH * kScRPW + KB * 12) * 4 <= kWarps * 2 * 16 * kScDC * 4, "refinement tables");
    constexpr int RPW = kScRPW, PSZ = sc_psz(QH);
    extern __shared__ __align__(128) uint8_t smem[];
    __shared__ __align__(16) FusedArgs s_args;
    __shared__ int s_item;
    __shared__ __align__(8) uint64_t s_bar;
    __shared__ int s_flag;
    __shared__ int s_rlo, s_rhi;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int g = lane >> 2, t4 = lane & 3;      // fragment row group and column pair
    const int mx = g & 3, my0 = g >> 2;          // this lane's fragment pixels m0 = g, m1 = g + 8
    const FusedArgs &a = s_args;
    if (tid == 0) mbar_init(&s_bar, 1);

    for (int iter = 0;; ++iter) {
        int tx = 0, ty = 0;
        const PairDesc *pd = claim_tile<kThreads>(single, pairs, items, nitems, counter, iter, s_args, s_item, tid, tx, ty);
        if (!pd) return;
        const int RP = a.ref_box_w;
        const ScLayout L = sc_layout(RB, a.m, RP, a.tgt_box_w, a.box_h);
        uint8_t *sref = smem + L.sref;
        uint8_t *stgt = smem + L.stgt;
        __half *cb16 = reinterpret_cast<__half *>(smem + L.cbuf);
        float *cb32 = reinterpret_cast<float *>(smem + L.cbuf);
        int *vband = reinterpret_cast<int *>(smem + L.escr);
        float *escr = reinterpret_cast<float *>(smem + L.escr);
        int2 *sstr = reinterpret_cast<int2 *>(smem + L.sstr);
        int2 *sstt = reinterpret_cast<int2 *>(smem + L.sstt);
        float *sI = reinterpret_cast<float *>(smem + L.sI);
        float4 *skxy = reinterpret_cast<float4 *>(smem + L.skxy);
        const int x0 = tx * TX, y0 = ty * TY;
        if (tid == 0) {
            s_rlo = 0x7fffffff;
            s_rhi = -1;
        }

        if (!stage_images(pd, a, sref, stgt, &s_bar, &s_flag, x0, y0, iter, tid)) return;

        const int rw = a.rw;
        // scaled reference intensities of the cost positions, exactly as k_fused stages them;
        // positions outside the image and the row padding get 1e18 (weight 0)
        for (int i = tid; i < QH * QWI; i += kThreads) {
            const int yq = i / QWI, xq = i - yq * QWI;
            const int ix = x0 - RB + xq, iy = y0 - RB + yq;
            float v = 1e18f;
            if (xq < QW && ix >= 0 && ix < a.W && iy >= 0 && iy < a.H)
                v = (float)sref[(yq + rw) * RP + a.ref_e + xq + rw] * a.iscale;
            sI[i] = v;
        }
        // -(K + 12) per (window row r, lane) in the A-fragment layout: pixels m0 = (mx, my),
        // m1 = (mx, my + 2); columns 2 t4 + {0, 1} (first float4) and 2 t4 + {8, 9} (second)
        for (int e = tid; e < NKS * 32; e += kThreads) {
            const int r = e >> 5, ln = e & 31, lg = ln >> 2, lt = ln & 3, lmx = lg & 3, lmy = lg >> 2;
            auto nk = [&](int col, int my) {
                const int dx = col - lmx, dy = r - my;
                return (dx >= 0 && dx <= 2 * RB && dy >= 0 && dy <= 2 * RB) ? -(a.K[dx * KB + dy] + (float)kScWSh)
                                                                             : 1e30f;
            };
            skxy[2 * e] = make_float4(nk(2 * lt, lmy), nk(2 * lt + 1, lmy), nk(2 * lt, lmy + 2), nk(2 * lt + 1, lmy + 2));
            skxy[2 * e + 1] =
                make_float4(nk(2 * lt + 8, lmy), nk(2 * lt + 9, lmy), nk(2 * lt + 8, lmy + 2), nk(2 * lt + 9, lmy + 2));
        }
        __syncthreads();

        // screening state of the lane's pixel in each patch pair (patch 2 pp + (lane >> 4),
        // pixel lane & 15): the running minimum of E16 and the candidate range
        float emin[NPP];
        int dlo[NPP], dhi[NPP];
#pragma unroll
        for (int i = 0; i < NPP; ++i) {
            emin[i] = __int_as_float(0x7f800000);
            dlo[i] = dhi[i] = 0;
        }
        float *scr = escr + warp * (2 * 16 * DC);

        for (int d0 = 0; d0 < (B2 ? 0 : a.D); d0 += DC) {
            // ---- costs of the chunk, 32 disparities, times 2^8, FP16, swizzled
            switch (rw) {
            case 1: cost_chunk<RB, DC, 1, __half, TX, TY, kThreads, 0, kScBand, true, kScCSh>(a, sref, stgt, cb16, vband, sstr, sstt, x0, y0, d0, tid); break;
            case 2: cost_chunk<RB, DC, 2, __half, TX, TY, kThreads, 0, kScBand, true, kScCSh>(a, sref, stgt, cb16, vband, sstr, sstt, x0, y0, d0, tid); break;
            case 3: cost_chunk<RB, DC, 3, __half, TX, TY, kThreads, 0, kScBand, true, kScCSh>(a, sref, stgt, cb16, vband, sstr, sstt, x0, y0, d0, tid); break;
            case 4: cost_chunk<RB, DC, 4, __half, TX, TY, kThreads, 0, kScBand, true, kScCSh>(a, sref, stgt, cb16, vband, sstr, sstt, x0, y0, d0, tid); break;
            default: cost_chunk<RB, DC, 5, __half, TX, TY, kThreads, 0, kScBand, true, kScCSh>(a, sref, stgt, cb16, vband, sstr, sstt, x0, y0, d0, tid); break;
            }
            // ---- screening aggregation, two patches at a time
#pragma unroll 1
            for (int pp = 0; pp < NPP; ++pp) {
                float2 nip[2][2];
                uint32_t brow[2][2];
                const float *irow[2];
                float acc[2][4][4];
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int P = warp * NPW + 2 * pp + h;
                    const int px0 = (P % NPX) * 4, py0 = (P / NPX) * 4;
                    const float ip0 = sI[(py0 + RB + my0) * QWI + px0 + RB + mx];
                    const float ip1 = sI[(py0 + RB + my0 + 2) * QWI + px0 + RB + mx];
                    nip[h][0] = make_float2(-ip0, -ip0);
                    nip[h][1] = make_float2(-ip1, -ip1);
                    // ldmatrix rows: lanes 8i..8i+7 name matrix i = (k half, unit): k slots
                    // 0..7 / 8..15 of the window row, 8-disparity units 2j + (lane >> 4)
                    const int kk = ((lane >> 3) & 1) * 8 + (lane & 7);
                    const int xq = min(px0 + kk, QW - 1);   // padding slots (zero weight) read a valid cost
                    const uint32_t pos = smem_addr(cb16 + ((size_t)py0 * QW + xq) * DC);
#pragma unroll
                    for (int j = 0; j < 2; ++j) brow[h][j] = pos + (uint32_t)(swz_unit<DC>(2 * j + (lane >> 4), xq) << 4);
                    irow[h] = sI + py0 * QWI + px0 + 2 * t4;
#pragma unroll
                    for (int nb = 0; nb < 4; ++nb)
#pragma unroll
                        for (int k = 0; k < 4; ++k) acc[h][nb][k] = 0.f;
                }
#pragma unroll
                for (int r = 0; r < NKS; ++r) {
                    const float4 klo = skxy[2 * (r * 32 + lane)], khi = skxy[2 * (r * 32 + lane) + 1];
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const float2 qlo = *reinterpret_cast<const float2 *>(irow[h] + r * QWI);
                        const float2 qhi = *reinterpret_cast<const float2 *>(irow[h] + r * QWI + 8);
                        // t = I_q - I_p; e' = t^2 - (K + 12); w16 = RN16(2^-e')
                        const float2 ta = __fadd2_rn(qlo, nip[h][0]), tb = __fadd2_rn(qlo, nip[h][1]);
                        const float2 tc = __fadd2_rn(qhi, nip[h][0]), td = __fadd2_rn(qhi, nip[h][1]);
                        const float2 ea = __ffma2_rn(ta, ta, make_float2(klo.x, klo.y));
                        const float2 eb = __ffma2_rn(tb, tb, make_float2(klo.z, klo.w));
                        const float2 ec = __ffma2_rn(tc, tc, make_float2(khi.x, khi.y));
                        const float2 ed = __ffma2_rn(td, td, make_float2(khi.z, khi.w));
                        uint32_t af[4];
                        af[0] = h2_rn(ex2_approx(-ea.x), ex2_approx(-ea.y));
                        af[1] = h2_rn(ex2_approx(-eb.x), ex2_approx(-eb.y));
                        af[2] = h2_rn(ex2_approx(-ec.x), ex2_approx(-ec.y));
                        af[3] = h2_rn(ex2_approx(-ed.x), ex2_approx(-ed.y));
                        const uint32_t roff = (uint32_t)(r * QW * DC * (int)sizeof(__half));
#pragma unroll
                        for (int j = 0; j < 2; ++j) {
                            uint32_t b0, b1, b2, b3;
                            ldsm_x4_t(brow[h][j] + roff, b0, b1, b2, b3);
                            X::mma(acc[h][2 * j], af, b0, b1);
                            X::mma(acc[h][2 * j + 1], af, b2, b3);
                        }
                    }
                }
                // the two 16 x 32 E blocks through the warp's scratch, one pixel per lane
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    float *sb = scr + h * 16 * DC;
#pragma unroll
                    for (int nb = 0; nb < 4; ++nb) {
                        const int u = 2 * nb + (t4 >> 1), o = 2 * (t4 & 1);
                        *reinterpret_cast<float2 *>(sb + g * DC + (sc_eunit(u, g) << 2) + o) =
                            make_float2(acc[h][nb][0], acc[h][nb][1]);
                        *reinterpret_cast<float2 *>(sb + (g + 8) * DC + (sc_eunit(u, g + 8) << 2) + o) =
                            make_float2(acc[h][nb][2], acc[h][nb][3]);
                    }
                }
                __syncwarp();
                {
                    const int m = lane & 15;
                    const float *er = scr + (lane >> 4) * 16 * DC + m * DC;
                    float e[DC];
#pragma unroll
                    for (int u = 0; u < DC / 4; ++u) {
                        const float4 v = *reinterpret_cast<const float4 *>(er + (sc_eunit(u, m) << 2));
                        e[4 * u] = v.x;
                        e[4 * u + 1] = v.y;
                        e[4 * u + 2] = v.z;
                        e[4 * u + 3] = v.w;
                    }
                    const int dn = min(DC, a.D - d0);
                    float cm = __int_as_float(0x7f800000);
#pragma unroll
                    for (int dd = 0; dd < DC; ++dd) {
                        if (dd >= dn) e[dd] = __int_as_float(0x7f800000);
                        cm = fminf(cm, e[dd]);
                    }
                    // the pair's state, selected with static indices (no local memory)
                    float em = emin[0];
#pragma unroll
                    for (int i = 1; i < NPP; ++i)
                        if (i == pp) em = emin[i];
                    const float nm = fminf(em, cm);
                    const float tn = sc_thr(nm);
                    uint32_t mask = 0;
#pragma unroll
                    for (int dd = 0; dd < DC; ++dd) mask |= (e[dd] <= tn) ? (1u << dd) : 0u;
                    const bool reset = mask && tn < em;   // the earlier range cannot hold d*
                    const int lo = d0 + __ffs(mask) - 1, hi = d0 + 31 - __clz(mask);
#pragma unroll
                    for (int i = 0; i < NPP; ++i)
                        if (i == pp) {
                            if (reset) dlo[i] = lo;
                            if (mask) dhi[i] = hi;
                            emin[i] = nm;
                        }
                }
                __syncwarp();
            }
            __syncthreads();
        }

        // ---- the tile's refinement range: [dlo - 1, dhi + 1] of every pixel inside the image,
        // clipped at df + 1, df = max(0, u + m - L + 1), where L is the shortest run of target
        // values equal to their row's column 0 over the rows v - m .. v + m (row table, .w).
        // For d >= df every target read behind pixel (u, v) falls at a column below L (or in
        // the replicate padding left of column 0) and returns its row's column-0 value, so each
        // block, its statistics and each cost c(q, d) are the same for all such d: E(p, d) =
        // E(p, df) exactly (the same terms in the same order).  The lowest d wins ties, so
        // d* <= df and d* + 1 stays inside the clipped range, and E(df) stands for the whole
        // tail in the smallest E over d != d*: the cut changes none of the outputs.
        int rlo[NPP], rhi[NPP];
        {
            int ulo = 0x7fffffff, uhi = -1;
#pragma unroll
            for (int pp = 0; pp < NPP; ++pp) {
                const int P = warp * NPW + 2 * pp + (lane >> 4), m = lane & 15;
                const int u = x0 + (P % NPX) * 4 + (m & 3), v = y0 + (P / NPX) * 4 + (m >> 2);
                const int lmin = (v < a.H) ? __ldg(&a.row_tab[v].w) : 1;
                const int cap = min(a.D - 1, max(0, u + a.m - lmin + 1) + 1);
                rlo[pp] = B2 ? 0 : max(dlo[pp] - 1, 0);
                rhi[pp] = min(B2 ? a.D - 1 : dhi[pp] + 1, cap);
                if (u < a.W && v < a.H) {
                    ulo = min(ulo, rlo[pp]);
                    uhi = max(uhi, rhi[pp]);
                } else {
                    rlo[pp] = 1;   // nothing to refine
                    rhi[pp] = 0;
                }
            }
            ulo = __reduce_min_sync(0xffffffffu, ulo);
            uhi = __reduce_max_sync(0xffffffffu, uhi);
            if (lane == 0 && uhi >= 0) {
                atomicMin(&s_rlo, ulo);
                atomicMax(&s_rhi, uhi);
            }
        }
        __syncthreads();
        const int ulo_t = s_rlo, uhi_t = s_rhi;

        // ---- refinement: k_fused's FP32 arithmetic and running WTA over the candidates, in
        // chunks of DCR disparities from the tile's lowest candidate.  The FP32 costs come from
        // the two-pass cost phase (the same integers and the same rounding as k_fused's costs).
        float best[NPP], bm1[NPP], bp1[NPP], prev[NPP], sec[B2 ? NPP : 1];
        int bd[NPP];
#pragma unroll
        for (int i = 0; i < NPP; ++i) {
            best[i] = __int_as_float(0x7f800000);
            bm1[i] = bp1[i] = prev[i] = best[i];
            if constexpr (B2) sec[i] = best[i];
            bd[i] = -1;
        }
        float *sIr = reinterpret_cast<float *>(smem + L.escr + kScRefOff);   // [QH][RPW]
        float *sKr = sIr + QH * RPW;                                           // [KB][12]
        for (int i = tid; i < QH * RPW; i += kThreads) {
            const int yq = i / RPW, xq = i - yq * RPW;
            sIr[i] = xq < QWI ? sI[yq * QWI + xq] : 1e18f;
        }
        for (int i = tid; i < KB * 12; i += kThreads) {
            const int dx = i / 12, dy = i - dx * 12;
            sKr[i] = dy < KB ? a.K[dx * KB + dy] : 0.f;
        }
        // (the first refinement chunk's cost phase synchronises before these are read)
        for (int cb = ulo_t; cb <= uhi_t; cb += DCR) {
            switch (rw) {
            case 1: cost_chunk<RB, DCR, 1, float, TX, TY, kThreads, 0, kScBand, false, 0, RPW, PSZ>(a, sref, stgt, cb32, vband, sstr, sstt, x0, y0, cb, tid); break;
            case 2: cost_chunk<RB, DCR, 2, float, TX, TY, kThreads, 0, kScBand, false, 0, RPW, PSZ>(a, sref, stgt, cb32, vband, sstr, sstt, x0, y0, cb, tid); break;
            case 3: cost_chunk<RB, DCR, 3, float, TX, TY, kThreads, 0, kScBand, false, 0, RPW, PSZ>(a, sref, stgt, cb32, vband, sstr, sstt, x0, y0, cb, tid); break;
            case 4: cost_chunk<RB, DCR, 4, float, TX, TY, kThreads, 0, kScBand, false, 0, RPW, PSZ>(a, sref, stgt, cb32, vband, sstr, sstt, x0, y0, cb, tid); break;
            default: cost_chunk<RB, DCR, 5, float, TX, TY, kThreads, 0, kScBand, false, 0, RPW, PSZ>(a, sref, stgt, cb32, vband, sstr, sstt, x0, y0, cb, tid); break;
            }
#pragma unroll
            for (int pp = 0; pp < NPP; ++pp) {
                const int lo = max(rlo[pp], cb), hi = min(rhi[pp], cb + DCR - 1);
                const int P = warp * NPW + 2 * pp + (lane >> 4), m = lane & 15;
                const int px = (P % NPX) * 4 + (m & 3), py = (P / NPX) * 4 + (m >> 2);
                const float ip = sIr[(py + RB) * RPW + px + RB];
                const float *ib = sIr + py * RPW + px;
                const float *cq = cb32 + py * RPW + px;   // plane 0; plane o at + o PSZ
                // three disparities per pass: d = g0, g0 + 1, g0 + 2 (those above hi discarded)
#pragma unroll 1
                for (int g0 = lo; g0 <= hi; g0 += 3) {
                    const int o0 = (g0 - cb) * PSZ, o1 = min(g0 - cb + 1, DCR - 1) * PSZ,
                              o2 = min(g0 - cb + 2, DCR - 1) * PSZ;
                    float e0 = 0.f, e1 = 0.f, e2 = 0.f;
#pragma unroll 1
                    for (int dx = 0; dx < KB; ++dx) {
                        float kr[12];
#pragma unroll
                        for (int k = 0; k < 3; ++k) {
                            const float4 q = *reinterpret_cast<const float4 *>(sKr + dx * 12 + 4 * k);
                            kr[4 * k] = q.x;
                            kr[4 * k + 1] = q.y;
                            kr[4 * k + 2] = q.z;
                            kr[4 * k + 3] = q.w;
                        }
#pragma unroll
                        for (int dy = 0; dy < KB; ++dy) {
                            const float t = ib[dy * RPW + dx] - ip;
                            const float w = ex2_approx(fmaf(-t, t, kr[dy]));
                            const float *c = cq + dy * RPW + dx;
                            e0 = fmaf(w, c[o0], e0);
                            e1 = fmaf(w, c[o1], e1);
                            e2 = fmaf(w, c[o2], e2);
                        }
                    }
                    const float ev[3] = {e0, e1, e2};
#pragma unroll
                    for (int j = 0; j < 3; ++j) {
                        const int d = g0 + j;
                        if (d > hi) break;
                        const float v = ev[j];
                        if (v < best[pp]) {
                            if constexpr (B2) sec[pp] = best[pp];
                            best[pp] = v;
                            bd[pp] = d;
                            bm1[pp] = prev[pp];
                        } else {
                            if constexpr (B2) sec[pp] = fminf(sec[pp], v);
                            if (d == bd[pp] + 1) bp1[pp] = v;
                        }
                        prev[pp] = v;
                    }
                }
            }
            __syncthreads();
        }
        // ---- epilogue: eq. (subpixel), add back s_i(v), validity from the row table (k_fused's)
#pragma unroll
        for (int pp = 0; pp < NPP; ++pp) {
            const int P = warp * NPW + 2 * pp + (lane >> 4), m = lane & 15;
            const int px = (P % NPX) * 4 + (m & 3), py = (P / NPX) * 4 + (m >> 2);
            const int u = x0 + px, v = y0 + py;
            if (u >= a.W || v >= a.H) continue;
            const int4 rt = __ldg(a.row_tab + v);   // {s_i(v), max s_i, min s_i over v +- m}
            float delta = 0.f;
            if (bd[pp] > 0 && bd[pp] < a.D - 1) {
                const float den = 2.f * bm1[pp] + 2.f * bp1[pp] - 4.f * best[pp];
                if (den > 0.f) delta = (bm1[pp] - bp1[pp]) / den;
            }
            const size_t o = (size_t)v * a.W + u;
            a.disp[o] = (float)bd[pp] + delta + (float)rt.x;
            if (a.wta) a.wta[o] = bd[pp];
            if (a.valid) {
                const int ulo = a.m + a.D - 1 + max(0, rt.y);
                const int uhi = a.W - 1 - a.m + min(0, rt.z);
                a.valid[o] = (uint8_t)(v >= a.m && v <= a.H - 1 - a.m && u >= ulo && u <= uhi);
            }
            if constexpr (B2) {
                // the skipped normaliser sum_q w(p,q), as k_fused sums it
                const float ip = sI[(py + RB) * QWI + px + RB];
                float ws = 0.f;
                for (int dx = 0; dx < KB; ++dx)
                    for (int dy = 0; dy < KB; ++dy) {
                        const float t = sI[(py + dy) * QWI + px + dx] - ip;
                        ws += ex2_approx(fmaf(-t, t, a.K[dx * KB + dy]));
                    }
                a.best2[2 * o] = best[pp] / ws;
                a.best2[2 * o + 1] = sec[pp] / ws;
            }
        }
    }  // tile loop
}

template <bool B2 = false>
FusedKernel pick_sc_rb(int rb)
{
    switch (rb) {
    case 0: return k_fused_sc<0, B2>;
    case 1: return k_fused_sc<1, B2>;
    case 2: return k_fused_sc<2, B2>;
    case 3: return k_fused_sc<3, B2>;
    case 4: return k_fused_sc<4, B2>;
    case 5: return k_fused_sc<5, B2>;
    }
    return nullptr;
}

}  // namespace sgb
