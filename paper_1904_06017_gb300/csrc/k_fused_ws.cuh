// k_fused_ws.cuh -- the warp-specialised form of the fused kernel (tile code kWsWC): producer
// warps compute the costs of chunk k + 1 into a second buffer while consumer warps aggregate
// chunk k, handing the two buffers over with named barriers.
#pragma once
#include "k_cost.cuh"

namespace sgb {

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

}  // namespace sgb
