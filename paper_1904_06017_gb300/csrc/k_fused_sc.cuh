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
// the tensor core's FP32 accumulation (at most 17 terms per k-step and 16 k-steps at bil = 13,
// each addition within 2^-23 of the running sum, truncating or rounding: 3.3e-5), k_fused's own
// chain of at most 169 FMAs (1.0e-5) and the ex2 / exponent roundings of the scaled weight
// (1e-5): 1.03e-3, taken as 1.1e-3; a (64, i.e. 6.1e-5 unscaled) covers FP16 subnormal weights
// and costs even if the tensor core flushed them.  Hence the FP32 argmin d* (lowest d on ties) satisfies
//     E16(d*) <= thr(min_d E16) = (min_d E16 + a) (1 + eps) / (1 - eps) + a,
// and so does every d that ties it.  Each pixel keeps the range [dlo, dhi] that holds every d
// with E16(d) <= thr(running minimum); a chunk whose minimum m makes thr(m) smaller than the
// previous minimum drops the earlier range (none of its disparities can satisfy the final test).
//
// Refinement.  After the last chunk the tile refines [dlo - 1, dhi + 1] of every pixel with
// k_fused's arithmetic (sc_refine): FP32 costs from the two-pass cost phase (the same integers
// and roundings as k_fused's), the weight ex2(fma(-t, t, K)), and the 121-term FMA chain in
// k_fused's order (window column outer, row inner), then k_fused's running WTA in increasing d.
// The winner and its two neighbours (the parabola of eq. subpixel) are therefore k_fused's
// values exactly.  With the best2 output (B2) every pixel refines all D disparities (a
// diagnostic path).
#pragma once
#include "k_fused_tc.cuh"

namespace sgb {

constexpr int kScDC = 32;       // disparities per screening chunk
constexpr int kScDCR = 8;       // disparities per FP32 refinement chunk
constexpr int kScRBand4 = 12;   // cost rows per band of a 4-disparity refinement chunk
constexpr int kScRBand8 = 8;    // cost rows per band of an 8-disparity refinement chunk
constexpr int kScRSeg = 3;      // cost columns per horizontal work item of the refinement chunks
constexpr int kScBand = 6;      // cost rows per band of the screening chunk's cost phase
constexpr int kScSeg = 6;       // cost columns per horizontal work item (6 rows x 7 segments x 8 quads = 336 items)
// Row length of the staged FP32 intensities (>= QW + 2, >= 28 + 16): 44 up to bil = 11 (the
// measured layout), 48 at bil = 13
__host__ __device__ constexpr int sc_qwi(int rb) { return rb >= 6 ? 48 : 44; }
// Refinement planes: rows of kScRPW entries and planes a multiple of 32 entries apart, so that
// a warp's 32 pixels of one row read 32 distinct banks whatever disparity each needs
constexpr int kScRPW = 44;
__host__ __device__ constexpr int sc_psz(int qh) { return (qh * kScRPW + 31) / 32 * 32; }
// Row length of the refinement's spatial-exponent table sKr: the 2 RB + 1 entries of a window
// column, padded to whole 16-byte rows
__host__ __device__ constexpr int sc_krw(int rb) { return (2 * rb + 1 + 3) / 4 * 4; }
constexpr int kScWSh = 12;      // weights scaled by 2^12 before rounding to FP16
constexpr int kScCSh = 8;       // costs scaled by 2^8
constexpr float kScEps = 1.1e-3f;
constexpr float kScAbs = 64.f;  // in the scaled units of E16 (2^20 x E32)
// (1 + eps) / (1 - eps), rounded up
constexpr float kScRho = (1.0f + kScEps) / (1.0f - kScEps) + 1e-6f;

constexpr int kScRefOff = 16384;     // bytes into escr: past the refinement's window sums (<= 10 KB)

__device__ __forceinline__ float sc_thr(float m) { return fmaf(m + kScAbs, kScRho, kScAbs); }

// Shared memory of the screened form (offsets from the 128-byte aligned dynamic base):
//   sref, stgt  image tiles (TMA), as in k_fused
//   cbuf   screening: [QH][QW][32] FP16 costs (16-byte units swizzled by bits 1..2 of the
//          column); refinement, in the same bytes: 4 planes of FP32 disparity pairs (float2
//          [QH][kScRPW], sc_psz(QH) entries apart), then the window statistics of a band
//   escr   the cost phase's vertical window sums ([band][CW][32] i32); the same bytes hold, in
//          the 16-bit form, two per-warp E blocks of the aggregation ([warp][2][16 pixels][32]
//          f32, 16-byte units swizzled by the pixel); after the screening the refinement's
//          vertical sums, and from kScRefOff on the intensities again as [QH][kScRPW] f32 and
//          the spatial exponents as [2 RB + 1][sc_krw(RB)] f32
//   sstr, sstt  window statistics of one band
//   sI     [QH][sc_qwi(RB)] f32  the reference intensities times sqrt(log2 e) / sigma1 of the cost
//          positions (1e18 outside the image, as in k_fused)
//   skxy   the row terms of the spatial exponent, (nKy(j), nKy(j - 2)) for j = -1 .. 3 + 2 RB
//          (float2)
//   sst    the screening state of every pixel of the tile ([TY][TX] float2: the running minimum
//          of E16, and the candidate range dlo | dhi << 16 as the bits of the second float)
struct ScLayout {
    size_t sref, stgt, cbuf, escr, sstr, sstt, sI, skxy, sst, total;
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
    L.skxy = align_up(L.sI + (size_t)QH * sc_qwi(rb) * 4, 16);
    L.sst = align_up(L.skxy + (size_t)(NKS + 2) * 8, 16);
    L.total = align_up(L.sst + (size_t)TY * TX * 8, 128);
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

// Packed pair of FP32 values rounded to the 16-bit type (lo in the low half).
template <typename T> __device__ __forceinline__ uint32_t pack_rn(float lo, float hi);
template <> __device__ __forceinline__ uint32_t pack_rn<__half>(float lo, float hi) { return h2_rn(lo, hi); }
template <> __device__ __forceinline__ uint32_t pack_rn<__nv_bfloat16>(float lo, float hi)
{
    uint32_t r;
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
    return r;
}

// ---- refinement of one tile (k_fused's FP32 arithmetic over each pixel's certified candidates)
//
// The range of pixel (u, v) is [dlo - 1, dhi + 1] (range_of(py, px) gives {dlo, dhi}; with B2
// every disparity), clipped at df + 1, df = max(0, u + m - L + 1), where L is the shortest run of
// target values equal to their row's column 0 over the rows v - m .. v + m (row table, .w).  For
// d >= df every target read behind the pixel falls at a column below L (or in the replicate
// padding left of column 0) and returns its row's column-0 value, so each block, its statistics
// and each cost c(q, d) are the same for all such d: E(p, d) = E(p, df) exactly (the same terms in
// the same order).  The lowest d wins ties, so d* <= df and d* + 1 stays inside the clipped range,
// and E(df) stands for the whole tail in the smallest E over d != d*: the cut changes none of the
// outputs.
//
// Each thread owns a column of RPY pixels (column lane, rows RPY warp ..), as the SIMT kernel's
// aggregation does: its loads serve every pixel of the column.  The tile's candidates are
// refined in chunks of DCR disparities (4 when they span at most 4) from the tile's lowest one;
// the FP32 costs come from the two-pass cost phase (the same integers and the same rounding as
// k_fused's costs), stored as planes of [QH][kScRPW] entries sc_psz(QH) apart.
//
// On entry: the tile's images are staged; sIr ([QH][kScRPW], the scaled reference intensities
// of the cost positions) and sKr ([KB][sc_krw(RB)], the spatial exponents K[dx][dy]) are written; *s_rlo
// = INT_MAX and *s_rhi = -1; and range_of's data are visible to every thread.  The function
// synchronises before it reads sIr and returns after the epilogue, without a final barrier.
// images_free() is called by every thread right after the barrier that ends the last chunk's
// cost phase: sref and stgt are not read after it.
template <int RB, bool B2, int NT, int DCR, int RKSEG, typename RangeOf, typename OnFree>
__device__ __forceinline__ void sc_refine(const FusedArgs &a, const uint8_t *sref, const uint8_t *stgt, float *cb32,
                                          int *vband, int2 *sstr, int2 *sstt, const float *sIr, const float *sKr,
                                          int x0, int y0, int tid, int *s_rlo, int *s_rhi, RangeOf range_of,
                                          OnFree images_free)
{
    constexpr int TX = tile_x(kScWC), TY = tile_y(kScWC);
    constexpr int KB = 2 * RB + 1, QH = TY + 2 * RB;
    constexpr int RPW = kScRPW, PSZ = sc_psz(QH);
    constexpr int NW = NT / 32, RPY = TY / NW;
    constexpr int KRW = sc_krw(RB);
    static_assert(TX == 32 && TY % NW == 0, "one warp per strip of RPY rows");
    static_assert(DCR == 4 || DCR == 8, "refinement chunks of 4 or 8 disparities");
    const int lane = tid & 31, warp = tid >> 5;
    const int px = lane, py0 = warp * RPY;
    int rlo[RPY], rhi[RPY];
    {
        int ulo = 0x7fffffff, uhi = -1;
#pragma unroll
        for (int i = 0; i < RPY; ++i) {
            const int u = x0 + px, v = y0 + py0 + i;
            rlo[i] = 1;   // nothing to refine outside the image
            rhi[i] = 0;
            if (u < a.W && v < a.H) {
                const int lmin = __ldg(&a.row_tab[v].w);
                const int cap = min(a.D - 1, max(0, u + a.m - lmin + 1) + 1);
                const int2 rg = B2 ? make_int2(0, 0) : range_of(py0 + i, px);
                rlo[i] = B2 ? 0 : max(rg.x - 1, 0);
                rhi[i] = min(B2 ? a.D - 1 : rg.y + 1, cap);
                ulo = min(ulo, rlo[i]);
                uhi = max(uhi, rhi[i]);
            }
        }
        ulo = __reduce_min_sync(0xffffffffu, ulo);
        uhi = __reduce_max_sync(0xffffffffu, uhi);
        if (lane == 0 && uhi >= 0) {
            atomicMin(s_rlo, ulo);
            atomicMax(s_rhi, uhi);
        }
    }
    __syncthreads();
    const int ulo_t = *s_rlo, uhi_t = *s_rhi;
    const int rw = a.rw;

    float best[RPY], bm1[RPY], bp1[RPY], prev[RPY], sec[B2 ? RPY : 1];
    int bd[RPY];
    float ip[RPY];
    int tlo = 0x7fffffff, thi = -1;   // the union of this thread's ranges
#pragma unroll
    for (int i = 0; i < RPY; ++i) {
        best[i] = __int_as_float(0x7f800000);
        bm1[i] = bp1[i] = prev[i] = best[i];
        if constexpr (B2) sec[i] = best[i];
        bd[i] = -1;
        ip[i] = sIr[(py0 + i + RB) * RPW + px + RB];
        if (rlo[i] <= rhi[i]) {
            tlo = min(tlo, rlo[i]);
            thi = max(thi, rhi[i]);
        }
    }
    const int dcr = (DCR == 4 || uhi_t - ulo_t < 4) ? 4 : DCR;
    const float2 *cb2 = reinterpret_cast<const float2 *>(cb32);
    for (int cb = ulo_t; cb <= uhi_t; cb += dcr) {
        if (DCR == 4 || dcr == 4) {
            switch (rw) {
            case 1: cost_chunk<RB, 4, 1, float, TX, TY, NT, 0, kScRBand4, false, 0, RPW, PSZ, RKSEG, true>(a, sref, stgt, cb32, vband, sstr, sstt, x0, y0, cb, tid); break;
            case 2: cost_chunk<RB, 4, 2, float, TX, TY, NT, 0, kScRBand4, false, 0, RPW, PSZ, RKSEG, true>(a, sref, stgt, cb32, vband, sstr, sstt, x0, y0, cb, tid); break;
            case 3: cost_chunk<RB, 4, 3, float, TX, TY, NT, 0, kScRBand4, false, 0, RPW, PSZ, RKSEG, true>(a, sref, stgt, cb32, vband, sstr, sstt, x0, y0, cb, tid); break;
            case 4: cost_chunk<RB, 4, 4, float, TX, TY, NT, 0, kScRBand4, false, 0, RPW, PSZ, RKSEG, true>(a, sref, stgt, cb32, vband, sstr, sstt, x0, y0, cb, tid); break;
            default: cost_chunk<RB, 4, 5, float, TX, TY, NT, 0, kScRBand4, false, 0, RPW, PSZ, RKSEG, true>(a, sref, stgt, cb32, vband, sstr, sstt, x0, y0, cb, tid); break;
            }
        } else {
            constexpr int D8 = DCR == 4 ? 4 : 8;
            switch (rw) {
            case 1: cost_chunk<RB, D8, 1, float, TX, TY, NT, 0, kScRBand8, false, 0, RPW, PSZ, RKSEG, true>(a, sref, stgt, cb32, vband, sstr, sstt, x0, y0, cb, tid); break;
            case 2: cost_chunk<RB, D8, 2, float, TX, TY, NT, 0, kScRBand8, false, 0, RPW, PSZ, RKSEG, true>(a, sref, stgt, cb32, vband, sstr, sstt, x0, y0, cb, tid); break;
            case 3: cost_chunk<RB, D8, 3, float, TX, TY, NT, 0, kScRBand8, false, 0, RPW, PSZ, RKSEG, true>(a, sref, stgt, cb32, vband, sstr, sstt, x0, y0, cb, tid); break;
            case 4: cost_chunk<RB, D8, 4, float, TX, TY, NT, 0, kScRBand8, false, 0, RPW, PSZ, RKSEG, true>(a, sref, stgt, cb32, vband, sstr, sstt, x0, y0, cb, tid); break;
            default: cost_chunk<RB, D8, 5, float, TX, TY, NT, 0, kScRBand8, false, 0, RPW, PSZ, RKSEG, true>(a, sref, stgt, cb32, vband, sstr, sstt, x0, y0, cb, tid); break;
            }
        }
        if (cb + dcr > uhi_t) images_free();   // the last chunk's cost phase has read the images
        // One pass per thread and chunk: disparities dw .. dw + 2 NPP - 1 from the pair below
        // the thread's lowest candidate in the chunk, NPP pairs (the warp's largest need; 2 or
        // 4).  Pairs past the chunk read its last pair (their sums are discarded), and so do the
        // threads with nothing to refine in the chunk.
        const int lo = max(tlo, cb), hi = min(thi, cb + dcr - 1);
        const int dw = lo <= hi ? cb + ((lo - cb) & ~1) : cb;
        const int need = lo <= hi ? (hi - dw) / 2 + 1 : 0;
        const int wneed = __reduce_max_sync(0xffffffffu, need);
        auto pass = [&](auto npp_c) {
            constexpr int NPP = decltype(npp_c)::value;
            int o[NPP];
#pragma unroll
            for (int k = 0; k < NPP; ++k) o[k] = min((dw - cb) / 2 + k, dcr / 2 - 1) * PSZ;
            float2 e[RPY][NPP];
#pragma unroll
            for (int i = 0; i < RPY; ++i)
#pragma unroll
                for (int k = 0; k < NPP; ++k) e[i][k] = make_float2(0.f, 0.f);
            const float *ib = sIr + py0 * RPW + px;
            const float2 *cq = cb2 + py0 * RPW + px;
#pragma unroll 1
            for (int dx = 0; dx < KB; ++dx) {
                float kr[KRW];
#pragma unroll
                for (int k = 0; k < KRW / 4; ++k) {
                    const float4 q = *reinterpret_cast<const float4 *>(sKr + dx * KRW + 4 * k);
                    kr[4 * k] = q.x;
                    kr[4 * k + 1] = q.y;
                    kr[4 * k + 2] = q.z;
                    kr[4 * k + 3] = q.w;
                }
                // neighbour rows of the column, in increasing order: for every pixel the window
                // rows come in k_fused's order (row inner, column outer); each FMA of a pair is
                // the scalar FMA of k_fused (same operands, one rounding)
#pragma unroll
                for (int r = 0; r < RPY + 2 * RB; ++r) {
                    const float iq = ib[r * RPW + dx];
                    float2 c[NPP];
#pragma unroll
                    for (int k = 0; k < NPP; ++k) c[k] = cq[r * RPW + dx + o[k]];
#pragma unroll
                    for (int i = 0; i < RPY; ++i) {
                        const int dy = r - i;
                        if (dy < 0 || dy > 2 * RB) continue;
                        const float t = iq - ip[i];
                        const float w = ex2_approx(fmaf(-t, t, kr[dy]));
                        const float2 w2 = make_float2(w, w);
#pragma unroll
                        for (int k = 0; k < NPP; ++k) e[i][k] = __ffma2_rn(w2, c[k], e[i][k]);
                    }
                }
            }
            // k_fused's running WTA, in increasing d
#pragma unroll
            for (int i = 0; i < RPY; ++i)
#pragma unroll
                for (int j = 0; j < 2 * NPP; ++j) {
                    const int d = dw + j;
                    if (d < rlo[i] || d > rhi[i] || d > hi) continue;
                    const float v = (j & 1) ? e[i][j >> 1].y : e[i][j >> 1].x;
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
        };
        if (wneed > 2) pass(std::integral_constant<int, 4>());
        else if (wneed > 0) pass(std::integral_constant<int, 2>());
        __syncthreads();
    }

    // ---- epilogue: eq. (subpixel), add back s_i(v), validity from the row table (k_fused's)
#pragma unroll
    for (int i = 0; i < RPY; ++i) {
        const int py = py0 + i;
        const int u = x0 + px, v = y0 + py;
        if (u >= a.W || v >= a.H) continue;
        const int4 rt = __ldg(a.row_tab + v);   // {s_i(v), max s_i, min s_i over v +- m, run}
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
            // the skipped normaliser sum_q w(p,q), as k_fused sums it
            const float ipp = sIr[(py + RB) * RPW + px + RB];
            float ws = 0.f;
            for (int dx = 0; dx < KB; ++dx)
                for (int dy = 0; dy < KB; ++dy) {
                    const float t = sIr[(py + dy) * RPW + px + dx] - ipp;
                    ws += ex2_approx(fmaf(-t, t, a.K[dx * KB + dy]));
                }
            a.best2[2 * o] = best[i] / ws;
            a.best2[2 * o + 1] = sec[i] / ws;
        }
    }
}

// ---- persistent tiles: the next work item is claimed while the current tile is still being
// worked on, and its images are staged into sref / stgt as soon as the tile's last cost phase
// has read them, so that the copies land during the refinement's evaluation and the epilogue.

// The pair and tile of work item `item` (a batch's work list, or one pair's tiles in order).
__device__ __forceinline__ const PairDesc *sc_decode(const PairDesc &single, const PairDesc *pairs,
                                                     const int2 *items, int item, int &tx, int &ty)
{
    if (pairs) {
        const int2 it = items[item];
        tx = it.y & 0xffff;
        ty = it.y >> 16;
        return pairs + it.x;
    }
    tx = item % single.ntx;
    ty = item / single.ntx;
    return &single;
}

// Waits for the images of the tile at (x0, y0), issuing their copies first unless an earlier
// call of sc_claim_ahead did (issued).  The wait is bounded as in stage_images, with the same
// fail-safe: false, with the status word set, when the copies did not land.
__device__ __forceinline__ bool sc_stage(const PairDesc *pd, const FusedArgs &a, uint8_t *sref, uint8_t *stgt,
                                         uint64_t *bar, int *flag, int x0, int y0, int iter, int tid, bool issued)
{
    if (tid == 0) {
        const bool stall = a.stall_test != 0;
        if (!issued) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            mbar_expect_tx(bar, (uint32_t)(a.box_h * (a.ref_box_w + a.tgt_box_w)));
            if (!stall) {
                tma_load_3d(sref, &pd->tmap_ref, 0, (x0 + a.ref_box_x) / 16, y0, bar);
                tma_load_3d(stgt, &pd->tmap_tgt, 0, x0 / 16, y0, bar);
            }
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

// Thread 0, once per tile, after a barrier that follows the tile's last read of sref / stgt:
// claims the next work item (*next) and, when its boxes fit the current ones (always within one
// pair), issues its image copies (*staged = 1).  Nothing is issued under the stall test hook.
__device__ __forceinline__ void sc_claim_ahead(const PairDesc &single, const PairDesc *pairs, const int2 *items,
                                               int nitems, int *counter, int item, const FusedArgs &a,
                                               uint8_t *sref, uint8_t *stgt, uint64_t *bar, int *next,
                                               int *claimed, int *staged, int tx_w, int ty_h)
{
    if (*claimed) return;
    *claimed = 1;
    *staged = 0;
    const int nx = pairs ? atomicAdd(counter, 1) : item + (int)gridDim.x;
    *next = nx;
    if (nx >= nitems || a.stall_test) return;
    int txn = 0, tyn = 0;
    const PairDesc *pn = sc_decode(single, pairs, items, nx, txn, tyn);
    const int bh = pn->a.box_h, rbw = pn->a.ref_box_w, tbw = pn->a.tgt_box_w;
    if (bh != a.box_h || rbw != a.ref_box_w || tbw > a.tgt_box_w || pn->a.stall_test) return;
    const int x0n = txn * tx_w, y0n = tyn * ty_h;
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    mbar_expect_tx(bar, (uint32_t)(bh * (rbw + tbw)));
    tma_load_3d(sref, &pn->tmap_ref, 0, (x0n + pn->a.ref_box_x) / 16, y0n, bar);
    tma_load_3d(stgt, &pn->tmap_tgt, 0, x0n / 16, y0n, bar);
    *staged = 1;
}

// MODE: kScScreened (the FP32 screened form), or kScPlain (the FP16 / BF16 storage form: the
// same tensor-core aggregation of the 16-bit costs with a running WTA on its sums, no
// refinement).  B2: the best2 output.  T: the 16-bit type of the costs and weights.
constexpr int kScScreened = 0, kScPlain = 1;

template <int RB, bool B2 = false, int MODE = kScScreened, typename T = __half>
__global__ void __launch_bounds__(kThreads, 1)
k_fused_sc(const __grid_constant__ PairDesc single, const PairDesc *__restrict__ pairs,
           const int2 *__restrict__ items, int nitems, int *__restrict__ counter)
{
    using X = TcOps<T>;
    constexpr bool PLAIN = MODE == kScPlain;
    constexpr int DC = kScDC, DCR = kScDCR;
    constexpr int TX = tile_x(kScWC), TY = tile_y(kScWC);
    constexpr int KB = 2 * RB + 1;
    constexpr int QH = TY + 2 * RB, QW = TX + 2 * RB;
    constexpr int QWI = sc_qwi(RB);
    constexpr int NKS = 4 + 2 * RB;              // k-steps: the window rows of a patch
    constexpr int NPX = TX / 4, NPY = TY / 4;    // patches of the tile
    constexpr int NPW = NPX * NPY / kWarps;      // patches per warp
    static_assert(RB <= kScMaxRB && NKS <= 16 && QW + 2 <= QWI,
                  "a window row spans at most 16 columns");
    static_assert((NPX * NPY) % kWarps == 0 && NPW % 2 == 0, "patches must split evenly over the warps");
    static_assert(kScRBand8 * (TX + 2 * (RB + kMaxRW)) * kScDCR * 4 <= kScRefOff &&
                      kScRBand4 * (TX + 2 * (RB + kMaxRW)) * 4 * 4 <= kScRefOff, "refinement window sums");
    // the refinement's band statistics sit in the cost buffer, past its FP32 planes
    static_assert(kScRBand8 <= kScRBand4, "the refinement statistics are sized for the taller band");
    static_assert((size_t)kScDCR * sc_psz(QH) * 4 + (size_t)kScRBand4 * (2 * QW + kScDCR - 1) * 8 <=
                      (size_t)QH * QW * kScDC * 2, "refinement statistics");
    static_assert(kScRefOff + (QH * kScRPW + KB * sc_krw(RB)) * 4 <= kScBand * (TX + 2 * RB) * kScDC * 4,
                  "refinement tables");
    constexpr int RPW = kScRPW, PSZ = sc_psz(QH);
    extern __shared__ __align__(128) uint8_t smem[];
    __shared__ __align__(16) FusedArgs s_args;
    __shared__ int s_item;
    __shared__ __align__(8) uint64_t s_bar;
    __shared__ int s_flag;
    __shared__ int s_rlo, s_rhi;
    __shared__ int s_next, s_claimed, s_staged;   // the work item claimed ahead, its copies issued
    __shared__ int s_dend;                        // the tile's screening chunks start below this

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int g = lane >> 2, t4 = lane & 3;      // fragment row group and column pair
    const int mx = g & 3, my0 = g >> 2;          // this lane's fragment pixels m0 = g, m1 = g + 8
    const FusedArgs &a = s_args;
    if (tid == 0) {
        mbar_init(&s_bar, 1);
        s_staged = 0;
    }

    for (int iter = 0;; ++iter) {
        // the work item: the first one claimed here, every later one claimed ahead (the barrier
        // also orders the previous tile's last reads of s_args before it is overwritten)
        if (tid == 0) {
            s_item = iter == 0 ? (pairs ? atomicAdd(counter, 1) : (int)blockIdx.x) : s_next;
            s_claimed = 0;
        }
        __syncthreads();
        const int item = s_item;
        if (item >= nitems) return;
        const bool issued = iter > 0 && s_staged;
        int tx = 0, ty = 0;
        const PairDesc *pd = sc_decode(single, pairs, items, item, tx, ty);
        {
            const int *src = reinterpret_cast<const int *>(&pd->a);
            int *dst = reinterpret_cast<int *>(&s_args);
            for (int i = tid; i < (int)(sizeof(FusedArgs) / 4); i += kThreads) dst[i] = src[i];
        }
        __syncthreads();
        const int RP = a.ref_box_w;
        const ScLayout L = sc_layout(RB, a.m, RP, a.tgt_box_w, a.box_h);
        uint8_t *sref = smem + L.sref;
        uint8_t *stgt = smem + L.stgt;
        T *cb16 = reinterpret_cast<T *>(smem + L.cbuf);
        float *cb32 = reinterpret_cast<float *>(smem + L.cbuf);
        int *vband = reinterpret_cast<int *>(smem + L.escr);
        float *escr = reinterpret_cast<float *>(smem + L.escr);
        int2 *sstr = reinterpret_cast<int2 *>(smem + L.sstr);
        int2 *sstt = reinterpret_cast<int2 *>(smem + L.sstt);
        float *sI = reinterpret_cast<float *>(smem + L.sI);
        const int x0 = tx * TX, y0 = ty * TY;
        if (tid == 0) {
            s_rlo = 0x7fffffff;
            s_rhi = -1;
        }
        if (!PLAIN && warp == 0) {
            // For d >= df = max(0, u + m - L + 1) every cost behind pixel (u, v) repeats its value at
            // df (L: the row table's shortest column-0 run over v +- m), so a chunk that starts past
            // the tile's largest df + 1 changes no candidate range (they are clipped at df + 1): the
            // screening stops before it.  (The 16-bit form's running WTA would take the same cut,
            // its values tying E(df), without best2; there the extra live state costs more.)
            int lm = 0x7fffffff;
            for (int v = y0 + lane; v < min(y0 + TY, a.H); v += 32) lm = min(lm, __ldg(&a.row_tab[v].w));
            lm = __reduce_min_sync(0xffffffffu, lm);
            if (lane == 0) s_dend = min(a.D, max(0, min(x0 + TX, a.W) - 1 + a.m - lm + 1) + 2);
        }

        if (!sc_stage(pd, a, sref, stgt, &s_bar, &s_flag, x0, y0, iter, tid, issued)) return;
        // called after a barrier that follows the tile's last read of sref / stgt
        auto images_free = [&]() {
            if (tid == 0)
                sc_claim_ahead(single, pairs, items, nitems, counter, item, a, sref, stgt, &s_bar, &s_next,
                               &s_claimed, &s_staged, TX, TY);
        };

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
        // spatial exponents, separable: -(K[dx][dy] + 12) = nKx(dx) + nKy(dy) with
        // nKx(i) = -(K[i][RB] + 12) and nKy(j) = -K[RB][j] (1e30 outside the window: weight 0).
        // The row terms as a table over j = r - my (the lane's first pixel row): (nKy(j), nKy(j - 2))
        float2 *sky = reinterpret_cast<float2 *>(smem + L.skxy);
        auto nky = [&](int j) { return (j >= 0 && j <= 2 * RB) ? -a.K[RB * KB + j] : 1e30f; };
        for (int j = tid; j < NKS + 2; j += kThreads) sky[j] = make_float2(nky(j - 1), nky(j - 3));
        if constexpr (!PLAIN) {
            float2 *sst0 = reinterpret_cast<float2 *>(smem + L.sst);
            for (int j = tid; j < TY * TX; j += kThreads) sst0[j] = make_float2(__int_as_float(0x7f800000), 0.f);
        }
        // this lane's column terms: columns 2 t4 + {0, 1} and 2 t4 + {8, 9} of a window row
        auto nkx = [&](int col) {
            const int i = col - mx;
            return (i >= 0 && i <= 2 * RB) ? -(a.K[i * KB + RB] + (float)kScWSh) : 1e30f;
        };
        const float2 nkx_lo = make_float2(nkx(2 * t4), nkx(2 * t4 + 1));
        const float2 nkx_hi = make_float2(nkx(2 * t4 + 8), nkx(2 * t4 + 9));
        __syncthreads();

        // Screening work: vertical segments of three patches (8 patch columns x 3 segments of 3
        // patch rows), two per warp.  The patches of a segment share their window rows: each
        // row's costs (ldmatrix) and intensities are read once for every patch that uses it.
        constexpr int NSEGR = NPY / 3;                // segments per patch column
        constexpr int NR3 = 8 + NKS;                  // window rows of a segment
        static_assert(NPY % 3 == 0 && NPX * NSEGR == 2 * kWarps, "two segments of three patches per warp");
        // the screening state of each pixel lives in sst between chunks (set before the barrier
        // above); a quad reads its two pixels' entries and its first lane writes them back
        float2 *sst = reinterpret_cast<float2 *>(smem + L.sst);
        const int hb = lane >> 4, m = lane & 15;
        // the plain form's running WTA (k_fused's rules on the 16-bit sums): per segment, state 0
        // is pixel m of patch hb, state 1 (lanes 0-15) pixel m of patch 2
        struct Wta {
            float best, bm1, bp1, prev, sec;
            int bd;
        };
        Wta ws[2][2];
#pragma unroll
        for (int si = 0; si < 2; ++si)
#pragma unroll
            for (int k = 0; k < 2; ++k) {
                const float inf = __int_as_float(0x7f800000);
                ws[si][k] = Wta{inf, inf, inf, inf, inf, -1};
            }

        const int dend = B2 ? 0 : s_dend;   // the screened form's bound (set before sc_stage's barrier)
        for (int d0 = 0; d0 < (PLAIN ? a.D : dend); d0 += DC) {
            // ---- costs of the chunk, 32 disparities, times 2^8, FP16, swizzled
            switch (rw) {
            case 1: cost_chunk<RB, DC, 1, T, TX, TY, kThreads, 0, kScBand, true, kScCSh, 0, 0, kScSeg>(a, sref, stgt, cb16, vband, sstr, sstt, x0, y0, d0, tid); break;
            case 2: cost_chunk<RB, DC, 2, T, TX, TY, kThreads, 0, kScBand, true, kScCSh, 0, 0, kScSeg>(a, sref, stgt, cb16, vband, sstr, sstt, x0, y0, d0, tid); break;
            case 3: cost_chunk<RB, DC, 3, T, TX, TY, kThreads, 0, kScBand, true, kScCSh, 0, 0, kScSeg>(a, sref, stgt, cb16, vband, sstr, sstt, x0, y0, d0, tid); break;
            case 4: cost_chunk<RB, DC, 4, T, TX, TY, kThreads, 0, kScBand, true, kScCSh, 0, 0, kScSeg>(a, sref, stgt, cb16, vband, sstr, sstt, x0, y0, d0, tid); break;
            default: cost_chunk<RB, DC, 5, T, TX, TY, kThreads, 0, kScBand, true, kScCSh, 0, 0, kScSeg>(a, sref, stgt, cb16, vband, sstr, sstt, x0, y0, d0, tid); break;
            }
            if constexpr (PLAIN)
                if (d0 + DC >= a.D) images_free();   // the aggregation and epilogue read no image
            const int dn = min(DC, a.D - d0);
#pragma unroll 1
            for (int si = 0; si < 2; ++si) {
                const int sg = warp + kWarps * si;
                const int px0 = (sg % NPX) * 4, pys = (sg / NPX) * 12;
                float2 nip[3][2];
#pragma unroll
                for (int i = 0; i < 3; ++i) {
                    const float ip0 = sI[(pys + 4 * i + RB + my0) * QWI + px0 + RB + mx];
                    const float ip1 = sI[(pys + 4 * i + RB + my0 + 2) * QWI + px0 + RB + mx];
                    nip[i][0] = make_float2(-ip0, -ip0);
                    nip[i][1] = make_float2(-ip1, -ip1);
                }
                // ldmatrix rows: lanes 8i..8i+7 name matrix i = (k half, unit): k slots 0..7 /
                // 8..15 of the window row, 8-disparity units 2j + (lane >> 4)
                const int kk = ((lane >> 3) & 1) * 8 + (lane & 7);
                const int xq = min(px0 + kk, QW - 1);   // padding slots (zero weight) read a valid cost
                const uint32_t pos = smem_addr(cb16 + ((size_t)pys * QW + xq) * DC);
                uint32_t brow[2];
#pragma unroll
                for (int j = 0; j < 2; ++j) brow[j] = pos + (uint32_t)(swz_unit<DC>(2 * j + (lane >> 4), xq) << 4);
                const float *irow = sI + pys * QWI + px0 + 2 * t4;
                float acc[3][4][4];
#pragma unroll
                for (int i = 0; i < 3; ++i)
#pragma unroll
                    for (int nb = 0; nb < 4; ++nb)
#pragma unroll
                        for (int k = 0; k < 4; ++k) acc[i][nb][k] = 0.f;
#pragma unroll
                for (int ra = 0; ra < NR3; ++ra) {
                    const float2 qlo = *reinterpret_cast<const float2 *>(irow + ra * QWI);
                    const float2 qhi = *reinterpret_cast<const float2 *>(irow + ra * QWI + 8);
                    uint32_t b[2][4];
                    const uint32_t roff = (uint32_t)(ra * QW * DC * (int)sizeof(__half));
#pragma unroll
                    for (int j = 0; j < 2; ++j) ldsm_x4_t(brow[j] + roff, b[j][0], b[j][1], b[j][2], b[j][3]);
#pragma unroll
                    for (int i = 0; i < 3; ++i) {
                        const int r = ra - 4 * i;             // this patch's window row
                        if (r < 0 || r >= NKS) continue;
                        const float2 ky = sky[r - my0 + 1];   // (nKy(r - my0), nKy(r - my0 - 2))
                        // t = I_q - I_p; e' = t^2 - (K + 12); w16 = RN16(2^-e')
                        const float2 ta = __fadd2_rn(qlo, nip[i][0]), tb = __fadd2_rn(qlo, nip[i][1]);
                        const float2 tc = __fadd2_rn(qhi, nip[i][0]), td = __fadd2_rn(qhi, nip[i][1]);
                        const float2 ea = __fadd2_rn(__ffma2_rn(ta, ta, nkx_lo), make_float2(ky.x, ky.x));
                        const float2 eb = __fadd2_rn(__ffma2_rn(tb, tb, nkx_lo), make_float2(ky.y, ky.y));
                        const float2 ec = __fadd2_rn(__ffma2_rn(tc, tc, nkx_hi), make_float2(ky.x, ky.x));
                        const float2 ed = __fadd2_rn(__ffma2_rn(td, td, nkx_hi), make_float2(ky.y, ky.y));
                        uint32_t af[4];
                        af[0] = pack_rn<T>(ex2_approx(-ea.x), ex2_approx(-ea.y));
                        af[1] = pack_rn<T>(ex2_approx(-eb.x), ex2_approx(-eb.y));
                        af[2] = pack_rn<T>(ex2_approx(-ec.x), ex2_approx(-ec.y));
                        af[3] = pack_rn<T>(ex2_approx(-ed.x), ex2_approx(-ed.y));
#pragma unroll
                        for (int j = 0; j < 2; ++j) {
                            X::mma(acc[i][2 * j], af, b[j][0], b[j][1]);
                            X::mma(acc[i][2 * j + 1], af, b[j][2], b[j][3]);
                        }
                    }
                }
                if constexpr (PLAIN) {
                    // two E blocks per warp: patches 0 and 1 (one pixel per lane), then patch 2
                    float *scr2 = escr + warp * (2 * 16 * DC);
                    auto put = [&](int i, int slot) {
                        float *sb = scr2 + slot * 16 * DC;
#pragma unroll
                        for (int nb = 0; nb < 4; ++nb) {
                            const int u = 2 * nb + (t4 >> 1), o = 2 * (t4 & 1);
                            *reinterpret_cast<float2 *>(sb + g * DC + (sc_eunit(u, g) << 2) + o) =
                                make_float2(acc[i][nb][0], acc[i][nb][1]);
                            *reinterpret_cast<float2 *>(sb + (g + 8) * DC + (sc_eunit(u, g + 8) << 2) + o) =
                                make_float2(acc[i][nb][2], acc[i][nb][3]);
                        }
                    };
                    auto run = [&](int slot, int k) {
                        const float *er = scr2 + slot * 16 * DC + m * DC;
                        float e[DC];
#pragma unroll
                        for (int u = 0; u < DC / 4; ++u) {
                            const float4 v = *reinterpret_cast<const float4 *>(er + (sc_eunit(u, m) << 2));
                            e[4 * u] = v.x;
                            e[4 * u + 1] = v.y;
                            e[4 * u + 2] = v.z;
                            e[4 * u + 3] = v.w;
                        }
                        Wta st = ws[0][k];
                        if (si == 1) st = ws[1][k];
                        float cmin = e[0];
#pragma unroll
                        for (int dd = 1; dd < DC; ++dd) cmin = fminf(cmin, e[dd]);
                        if (dn == DC && !(cmin < st.best)) {
                            // no new best in this full chunk: the walk below would only set E(d* + 1)
                            // when d* is the previous chunk's last disparity, fold the chunk into
                            // the smallest E over d != d*, and leave its last value as prev
                            if (st.bd == d0 - 1) st.bp1 = e[0];
                            if constexpr (B2) st.sec = fminf(st.sec, cmin);
                            st.prev = e[DC - 1];
                        } else {
#pragma unroll
                            for (int dd = 0; dd < DC; ++dd) {
                                if (dd >= dn) break;
                                const float v = e[dd];
                                const int d = d0 + dd;
                                if (v < st.best) {
                                    if constexpr (B2) st.sec = st.best;
                                    st.best = v;
                                    st.bd = d;
                                    st.bm1 = st.prev;
                                } else {
                                    if constexpr (B2) st.sec = fminf(st.sec, v);
                                    if (d == st.bd + 1) st.bp1 = v;
                                }
                                st.prev = v;
                            }
                        }
                        if (si == 0) ws[0][k] = st;
                        else ws[1][k] = st;
                    };
                    // A full chunk in which no pixel of the warp gets a new best skips the E
                    // blocks: each pixel's minimum over the chunk comes from its quad (lane (g, t4)
                    // holds disparities 8 nb + 2 t4 + {0, 1} of pixels g and g + 8), and the lane
                    // that keeps the pixel's WTA state (pixel m = g + 8 h: state 0 of patch hb,
                    // state 1 of patch 2) receives it, and the chunk's first value E(d0) (lane 4 g,
                    // nb = 0) and last value E(d0 + 31) (lane 4 g + 3, nb = 3), by shuffles; the
                    // state then takes what run() would give it for such a chunk
                    bool walk = dn < DC;
                    if (!walk) {
                        float c[3][2];
#pragma unroll
                        for (int i = 0; i < 3; ++i)
#pragma unroll
                            for (int h = 0; h < 2; ++h) {
                                float v = fminf(acc[i][0][2 * h], acc[i][0][2 * h + 1]);
#pragma unroll
                                for (int nb = 1; nb < 4; ++nb) v = fminf(v, fminf(acc[i][nb][2 * h], acc[i][nb][2 * h + 1]));
                                v = fminf(v, __shfl_xor_sync(0xffffffffu, v, 1));
                                c[i][h] = fminf(v, __shfl_xor_sync(0xffffffffu, v, 2));
                            }
                        const int src = 4 * (m & 7), hm = m >> 3;
                        auto pick = [&](const float (&x)[3][2], int patch) {
                            // x[patch][hm] of the shuffled values, with static indices
                            const float a0 = hm ? x[0][1] : x[0][0], a1 = hm ? x[1][1] : x[1][0];
                            const float a2 = hm ? x[2][1] : x[2][0];
                            return patch == 2 ? a2 : patch == 1 ? a1 : a0;
                        };
                        float xm[3][2];
#pragma unroll
                        for (int i = 0; i < 3; ++i)
#pragma unroll
                            for (int h = 0; h < 2; ++h) xm[i][h] = __shfl_sync(0xffffffffu, c[i][h], src);
                        Wta s0 = ws[0][0], s1 = ws[0][1];
                        if (si == 1) {
                            s0 = ws[1][0];
                            s1 = ws[1][1];
                        }
                        const float m0 = pick(xm, hb), m1 = pick(xm, 2);
                        walk = __any_sync(0xffffffffu, m0 < s0.best || (hb == 0 && m1 < s1.best));
                        if (!walk) {
                            float xl[3][2], xf[3][2];
#pragma unroll
                            for (int i = 0; i < 3; ++i)
#pragma unroll
                                for (int h = 0; h < 2; ++h) {
                                    xl[i][h] = __shfl_sync(0xffffffffu, acc[i][3][2 * h + 1], src + 3);
                                    xf[i][h] = 0.f;
                                }
                            if (__any_sync(0xffffffffu, s0.bd == d0 - 1 || (hb == 0 && s1.bd == d0 - 1))) {
#pragma unroll
                                for (int i = 0; i < 3; ++i)
#pragma unroll
                                    for (int h = 0; h < 2; ++h) xf[i][h] = __shfl_sync(0xffffffffu, acc[i][0][2 * h], src);
                            }
                            if (s0.bd == d0 - 1) s0.bp1 = pick(xf, hb);
                            if constexpr (B2) s0.sec = fminf(s0.sec, m0);
                            s0.prev = pick(xl, hb);
                            if (hb == 0) {
                                if (s1.bd == d0 - 1) s1.bp1 = pick(xf, 2);
                                if constexpr (B2) s1.sec = fminf(s1.sec, m1);
                                s1.prev = pick(xl, 2);
                            }
                            if (si == 0) {
                                ws[0][0] = s0;
                                ws[0][1] = s1;
                            } else {
                                ws[1][0] = s0;
                                ws[1][1] = s1;
                            }
                        }
                    }
                    if (walk) {
                        put(0, 0);
                        put(1, 1);
                        __syncwarp();
                        run(hb, 0);
                        __syncwarp();
                        put(2, 0);
                        __syncwarp();
                        if (hb == 0) run(0, 1);
                        __syncwarp();
                    }
                } else {
                    // the screening update, straight from the fragments: lane (g, t4) holds
                    // disparities 8 nb + 2 t4 + {0, 1} (nb = 0..3) of pixels g and g + 8, and the
                    // four lanes of a quad hold all 32 disparities of the same two pixels
#pragma unroll
                    for (int i = 0; i < 3; ++i) {
#pragma unroll
                        for (int h = 0; h < 2; ++h) {
                            float v[8];
#pragma unroll
                            for (int nb = 0; nb < 4; ++nb) {
                                v[2 * nb] = acc[i][nb][2 * h];
                                v[2 * nb + 1] = acc[i][nb][2 * h + 1];
                            }
                            if (dn < DC) {   // the last chunk of a search range off the chunk grid
#pragma unroll
                                for (int j = 0; j < 8; ++j)
                                    if (8 * (j >> 1) + 2 * t4 + (j & 1) >= dn) v[j] = __int_as_float(0x7f800000);
                            }
                            float cm = v[0];
#pragma unroll
                            for (int j = 1; j < 8; ++j) cm = fminf(cm, v[j]);
                            cm = fminf(cm, __shfl_xor_sync(0xffffffffu, cm, 1));
                            cm = fminf(cm, __shfl_xor_sync(0xffffffffu, cm, 2));
                            // the pixel's state.  A chunk whose minimum lies above thr(running
                            // minimum) changes neither (every E16 of it fails the test, and the
                            // minimum stays): a warp with no such pixel skips the update
                            const int pidx = ((sg / NPX) * 12 + 4 * i + my0 + 2 * h) * TX + px0 + mx;
                            const float2 sv = sst[pidx];
                            const float em = sv.x;
                            if (!__any_sync(0xffffffffu, cm <= sc_thr(em))) continue;
                            const float nm = fminf(em, cm);
                            const float tn = sc_thr(nm);
                            uint32_t mk = 0;
#pragma unroll
                            for (int j = 0; j < 8; ++j) mk |= (v[j] <= tn) ? (1u << (8 * (j >> 1) + (j & 1))) : 0u;
                            mk <<= 2 * t4;
                            mk |= __shfl_xor_sync(0xffffffffu, mk, 1);
                            mk |= __shfl_xor_sync(0xffffffffu, mk, 2);
                            const bool reset = mk && tn < em;   // the earlier range cannot hold d*
                            const int lo = d0 + __ffs(mk) - 1, hi = d0 + 31 - __clz(mk);
                            int r = __float_as_int(sv.y);
                            if (reset) r = (r & ~0xffff) | lo;
                            if (mk) r = (r & 0xffff) | (hi << 16);
                            if (t4 == 0) sst[pidx] = make_float2(nm, __int_as_float(r));
                        }
                    }
                }
            }
            // The 16-bit form's E blocks share escr with the next cost phase's window sums.  The
            // screened form's aggregation reads nothing the next cost phase writes before its
            // first barrier (window sums, band statistics), so its fast warps go on to that
            // phase; the barrier there orders every read of this chunk's costs before the new
            // ones are stored.
            if constexpr (PLAIN) __syncthreads();
        }
        if constexpr (!PLAIN) __syncthreads();   // every pixel's screening state is final

        if constexpr (PLAIN) {
            // ---- epilogue of the plain form: eq. (subpixel), add back s_i(v), validity
#pragma unroll
            for (int si = 0; si < 2; ++si)
#pragma unroll
                for (int k = 0; k < 2; ++k) {
                    if (k == 1 && hb) continue;
                    const int sg = warp + kWarps * si, patch = k ? 2 : hb;
                    const int px = (sg % NPX) * 4 + (m & 3), py = (sg / NPX) * 12 + 4 * patch + (m >> 2);
                    const int u = x0 + px, v = y0 + py;
                    if (u >= a.W || v >= a.H) continue;
                    const Wta &st = ws[si][k];
                    const int4 rt = __ldg(a.row_tab + v);
                    float delta = 0.f;
                    if (st.bd > 0 && st.bd < a.D - 1) {
                        const float den = 2.f * st.bm1 + 2.f * st.bp1 - 4.f * st.best;
                        if (den > 0.f) delta = (st.bm1 - st.bp1) / den;
                    }
                    const size_t o = (size_t)v * a.W + u;
                    a.disp[o] = (float)st.bd + delta + (float)rt.x;
                    if (a.wta) a.wta[o] = st.bd;
                    if (a.valid) {
                        const int ulo = a.m + a.D - 1 + max(0, rt.y);
                        const int uhi = a.W - 1 - a.m + min(0, rt.z);
                        a.valid[o] = (uint8_t)(v >= a.m && v <= a.H - 1 - a.m && u >= ulo && u <= uhi);
                    }
                    if constexpr (B2) {
                        // the skipped normaliser in FP32 (the sums carry the factor 2^20)
                        const float ipp = sI[(py + RB) * QWI + px + RB];
                        float wsum = 0.f;
                        for (int dx = 0; dx < KB; ++dx)
                            for (int dy = 0; dy < KB; ++dy) {
                                const float t = sI[(py + dy) * QWI + px + dx] - ipp;
                                wsum += ex2_approx(fmaf(-t, t, a.K[dx * KB + dy]));
                            }
                        const float sc = 1.f / (float)(1 << (kScWSh + kScCSh));
                        a.best2[2 * o] = st.best * sc / wsum;
                        a.best2[2 * o + 1] = st.sec * sc / wsum;
                    }
                }
            __syncthreads();
            images_free();   // (claimed already, unless the chunk loop did not run)
            continue;        // the next tile
        }

        // ---- refinement of the candidates
        // the intensities on the refinement's row pitch: sI itself where the pitches agree
        float *sIc = reinterpret_cast<float *>(smem + L.escr + kScRefOff);   // [QH][RPW]
        float *sKr = sIc + QH * RPW;                                           // [KB][sc_krw(RB)]
        if constexpr (QWI != RPW) {
            for (int i = tid; i < QH * RPW; i += kThreads) {
                const int yq = i / RPW, xq = i - yq * RPW;
                sIc[i] = xq < QWI ? sI[yq * QWI + xq] : 1e18f;
            }
        }
        const float *sIr = QWI == RPW ? sI : sIc;
        for (int i = tid; i < KB * sc_krw(RB); i += kThreads) {
            const int dx = i / sc_krw(RB), dy = i - dx * sc_krw(RB);
            sKr[i] = dy < KB ? a.K[dx * KB + dy] : 0.f;
        }
        int2 *rstr = reinterpret_cast<int2 *>(cb32 + (size_t)DCR * PSZ);   // [kScRBand4][QW]
        int2 *rstt = rstr + kScRBand4 * QW;                                  // [kScRBand4][QW + DCR - 1]
        sc_refine<RB, B2, kThreads, DCR, kScRSeg>(a, sref, stgt, cb32, vband, rstr, rstt, sIr, sKr, x0, y0, tid, &s_rlo, &s_rhi,
                                         [&](int py, int px) {
                                             const int r = __float_as_int(sst[py * TX + px].y);
                                             return make_int2(r & 0xffff, r >> 16);
                                         },
                                         images_free);
        __syncthreads();
        images_free();   // (claimed already, unless the tile had no candidates to refine)
    }  // tile loop
}

template <bool B2 = false, int MODE = kScScreened, typename T = __half>
FusedKernel pick_sc_rb(int rb)
{
    switch (rb) {
    case 0: return k_fused_sc<0, B2, MODE, T>;
    case 1: return k_fused_sc<1, B2, MODE, T>;
    case 2: return k_fused_sc<2, B2, MODE, T>;
    case 3: return k_fused_sc<3, B2, MODE, T>;
    case 4: return k_fused_sc<4, B2, MODE, T>;
    case 5: return k_fused_sc<5, B2, MODE, T>;
    case 6: return k_fused_sc<6, B2, MODE, T>;   // bil = 13: a window row fills the 16 k-slots
    }
    return nullptr;
}

}  // namespace sgb
