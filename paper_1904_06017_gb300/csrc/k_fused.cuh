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
#include "k_cost.cuh"

namespace sgb {

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

}  // namespace sgb
