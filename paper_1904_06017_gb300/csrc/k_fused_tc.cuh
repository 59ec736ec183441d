// k_fused_tc.cuh -- the fused kernel with tensor-core aggregation, for FP16 / BF16 cost
// storage: matching cost (eq. c), bilateral aggregation (eq. omega_s, eq. fbs), winner-take-all
// and the parabola step (eq. subpixel), §3.2.
//
// The cost phase is k_fused's (cost_chunk), 16 disparities per chunk, stored as FP16 / BF16 in
// a swizzled layout.  The aggregation of a chunk,
//     E(p, d) = sum_q w(p, q) c(q, d),
// is a banded matrix product, computed per 4 x 4 patch of pixels with mma.sync m16n8k16
// (FP16 or BF16 operands, FP32 accumulators):
//   M = the 16 pixels of the patch (m = 4 my + mx), N = 8 disparities, and one k-step per row
//       of the patch's window (4 + 2 RB rows), K = the 4 + 2 RB cost columns that row spans,
//       padded to 16 with zero weights;
//   A = the bilateral weights, generated in registers in the fragment layout:
//       w = 2^(Kx(dx) + Ky(dy) - s^2 (I_q - I_p)^2), zero outside the k x k window; Kx + Ky
//       per (window row, lane) from a shared table, the rest of the exponent in packed 16-bit
//       arithmetic on the exact integer intensity difference, the power by ex2.approx on the
//       packed pair;
//   B = the costs, gathered by ldmatrix.trans: every lane names one 16-byte row (a cost
//       position, 8 disparities), so a k-step's 16 positions are read in one instruction.
// The two patches of a pair advance k-step by k-step together.  Their accumulated blocks E
// (16 pixels x 16 disparities each) go through a per-warp scratch to the running WTA, one
// pixel per lane, disparities in increasing order (lowest d wins ties).
// The weights are rounded to the storage type and the weight normaliser is skipped, as in
// k_fused (a positive per-pixel factor changes neither the argmin nor the parabola step).
#pragma once
#include "k_cost.cuh"

namespace sgb {

constexpr int kTcDC = 16;      // disparities per chunk
constexpr int kTcQWI = 76;     // row length of the staged intensities (>= TX + 2 RB and >= 60 + 16)
constexpr float kTcFar = 30000.f;    // intensity of positions outside the image: its squared
                                     // difference drives the exponent to -inf (weight 0)
constexpr float kTcOff = -20000.f;   // spatial exponent outside the window (weight 0)
// cost rows per band of the cost phase: 12 where shared memory allows (half the barriers of 6)
__host__ __device__ constexpr int tc_band(int rb) { return rb <= 5 ? 12 : 6; }

// Shared memory of the tensor-core form (offsets from the 128-byte aligned dynamic base):
//   sref, stgt  image tiles (TMA), as in k_fused
//   cbuf   [QH][QW][16] T  the chunk's costs, 16-byte halves swizzled by bit 2 of the column
//   vband  [band][CW][16] i32 vertical window sums of the cost phase; the same bytes hold the
//          per-warp E blocks of the aggregation ([warp][2][16][16] f32)
//   sstr, sstt  window statistics of one band (band = tc_band(RB) cost rows)
//   sI     [QH][kTcQWI] T  raw reference intensities of the cost positions
//   skxy   [4 + 2 RB][32] uint4  spatial exponents Kx + Ky in the A-fragment layout, per window
//          row and lane (four packed pairs: fragment registers 0..3)
struct TcLayout {
    size_t sref, stgt, cbuf, vband, sstr, sstt, sI, skxy, total;
};

__host__ __device__ inline TcLayout tc_layout(int rb, int m, int ref_box_w, int tgt_box_w, int box_h, int esize)
{
    TcLayout L;
    const int TX = tile_x(kTcWC), TY = tile_y(kTcWC);
    const int QH = TY + 2 * rb, QW = TX + 2 * rb, CW = TX + 2 * m;
    const int band = tc_band(rb);
    const size_t vb = (size_t)band * CW * kTcDC * 4, eb = (size_t)kWarps * 2 * 256 * 4;
    L.sref = 0;
    L.stgt = align_up((size_t)box_h * ref_box_w, 128);
    L.cbuf = align_up(L.stgt + (size_t)box_h * tgt_box_w, 128);
    L.vband = align_up(L.cbuf + (size_t)QH * QW * kTcDC * esize, 128);
    L.sstr = align_up(L.vband + (vb > eb ? vb : eb), 16);
    L.sstt = align_up(L.sstr + (size_t)band * QW * 8, 16);
    L.sI = align_up(L.sstt + (size_t)band * (QW + kTcDC - 1) * 8, 16);
    L.skxy = align_up(L.sI + (size_t)QH * kTcQWI * esize, 16);
    L.total = align_up(L.skxy + (size_t)(4 + 2 * rb) * 32 * 16, 128);
    return L;
}

// Packed 16-bit operations of one storage type.
template <typename T> struct TcOps;
template <> struct TcOps<__half> {
    using T2 = __half2;
    static __device__ __forceinline__ T2 pair(float lo, float hi) { return __floats2half2_rn(lo, hi); }
    static __device__ __forceinline__ T2 dup(__half v) { return __half2half2(v); }
    static __device__ __forceinline__ __half from(float v) { return __float2half_rn(v); }
    static __device__ __forceinline__ uint32_t ex2(T2 x)
    {
        uint32_t y;
        asm("ex2.approx.f16x2 %0, %1;" : "=r"(y) : "r"(*reinterpret_cast<uint32_t *>(&x)));
        return y;
    }
    static __device__ __forceinline__ void mma(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1)
    {
        asm("mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
            "{%0, %1, %2, %3};"
            : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
            : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
    }
};
template <> struct TcOps<__nv_bfloat16> {
    using T2 = __nv_bfloat162;
    static __device__ __forceinline__ T2 pair(float lo, float hi) { return __floats2bfloat162_rn(lo, hi); }
    static __device__ __forceinline__ T2 dup(__nv_bfloat16 v) { return __bfloat162bfloat162(v); }
    static __device__ __forceinline__ __nv_bfloat16 from(float v) { return __float2bfloat16_rn(v); }
    static __device__ __forceinline__ uint32_t ex2(T2 x)
    {
        uint32_t y;
        asm("ex2.approx.ftz.bf16x2 %0, %1;" : "=r"(y) : "r"(*reinterpret_cast<uint32_t *>(&x)));
        return y;
    }
    static __device__ __forceinline__ void mma(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1)
    {
        asm("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
            "{%0, %1, %2, %3};"
            : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
            : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
    }
};

// Four 8 x 8 b16 matrices, transposed, from the 16-byte rows whose shared addresses lanes
// 8i .. 8i+7 give for matrix i.
__device__ __forceinline__ void ldsm_x4_t(uint32_t addr, uint32_t &r0, uint32_t &r1, uint32_t &r2, uint32_t &r3)
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0, %1, %2, %3}, [%4];"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(addr));
}

// Swizzle of a 16 x 16 FP32 E block: 16-byte unit u of pixel row m sits at unit u ^ f(m), so
// that both the fragment-layout stores (8 bytes, two rows per bank group) and the per-pixel
// LDS.128 reads are free of bank conflicts.
__device__ __forceinline__ int tc_eswz(int m) { return (m & 2) | ((m >> 2) & 1); }

// B2: also track the smallest E over d != d* and write best2 (a separate instantiation).
template <int RB, typename T, bool B2 = false>
__global__ void __launch_bounds__(kThreads, 1)
k_fused_tc(const __grid_constant__ PairDesc single, const PairDesc *__restrict__ pairs,
           const int2 *__restrict__ items, int nitems, int *__restrict__ counter)
{
    using X = TcOps<T>;
    using T2 = typename X::T2;
    constexpr int DC = kTcDC;
    constexpr int TX = tile_x(kTcWC), TY = tile_y(kTcWC);
    constexpr int KB = 2 * RB + 1;
    constexpr int QH = TY + 2 * RB, QW = TX + 2 * RB;
    constexpr int QWI = kTcQWI;
    constexpr int NKS = 4 + 2 * RB;              // k-steps: the window rows of a patch
    constexpr int NPX = TX / 4, NPY = TY / 4;    // patches of the tile
    constexpr int NPW = NPX * NPY / kWarps;      // patches per warp
    constexpr int NPP = NPW / 2;                 // handled two at a time
    static_assert(NKS <= 16 && QW <= QWI, "a window row spans at most 16 cost columns");
    static_assert((NPX * NPY) % kWarps == 0 && NPW % 2 == 0, "patches must split evenly over the warps");
    extern __shared__ __align__(128) uint8_t smem[];
    __shared__ __align__(16) FusedArgs s_args;
    __shared__ int s_item;
    __shared__ __align__(8) uint64_t s_bar;
    __shared__ int s_flag;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int g = lane >> 2, t4 = lane & 3;      // fragment row group and column pair
    const int mx = g & 3, my0 = g >> 2;          // this lane's pixels m0 = g, m1 = g + 8
    const FusedArgs &a = s_args;
    if (tid == 0) mbar_init(&s_bar, 1);

    for (int iter = 0;; ++iter) {
        int tx = 0, ty = 0;
        const PairDesc *pd = claim_tile<kThreads>(single, pairs, items, nitems, counter, iter, s_args, s_item, tid, tx, ty);
        if (!pd) return;
        const int RP = a.ref_box_w;
        const TcLayout L = tc_layout(RB, a.m, RP, a.tgt_box_w, a.box_h, (int)sizeof(T));
        uint8_t *sref = smem + L.sref;
        uint8_t *stgt = smem + L.stgt;
        T *cbuf = reinterpret_cast<T *>(smem + L.cbuf);
        int *vband = reinterpret_cast<int *>(smem + L.vband);
        float *escr = reinterpret_cast<float *>(smem + L.vband);
        int2 *sstr = reinterpret_cast<int2 *>(smem + L.sstr);
        int2 *sstt = reinterpret_cast<int2 *>(smem + L.sstt);
        T *sI = reinterpret_cast<T *>(smem + L.sI);
        uint4 *skxy = reinterpret_cast<uint4 *>(smem + L.skxy);
        const int x0 = tx * TX, y0 = ty * TY;

        if (!stage_images(pd, a, sref, stgt, &s_bar, &s_flag, x0, y0, iter, tid)) return;

        const int rw = a.rw;
        // raw reference intensities of the cost positions (exact in both 16-bit types);
        // positions outside the image and the row padding get kTcFar
        for (int i = tid; i < QH * QWI; i += kThreads) {
            const int yq = i / QWI, xq = i - yq * QWI;
            const int ix = x0 - RB + xq, iy = y0 - RB + yq;
            float v = kTcFar;
            if (xq < QW && ix >= 0 && ix < a.W && iy >= 0 && iy < a.H)
                v = (float)sref[(yq + rw) * RP + a.ref_e + xq + rw];
            sI[i] = X::from(v);
        }
        // spatial exponents in the fragment layout, per (window row r, lane): the four packed
        // pairs of fragment registers 0..3 (pixel m0 / m1, columns 2 t4 + {0,1} / + {8,9})
        for (int e = tid; e < NKS * 32; e += kThreads) {
            const int r = e >> 5, ln = e & 31, lg = ln >> 2, lt = ln & 3, lmx = lg & 3, lmy = lg >> 2;
            auto kx = [&](int dx) { return (dx >= 0 && dx <= 2 * RB) ? a.K[dx * KB + RB] : kTcOff; };
            auto ky = [&](int dy) { return (dy >= 0 && dy <= 2 * RB) ? a.K[RB * KB + dy] : kTcOff; };
            const float xl0 = kx(2 * lt - lmx), xl1 = kx(2 * lt + 1 - lmx);
            const float xh0 = kx(2 * lt + 8 - lmx), xh1 = kx(2 * lt + 9 - lmx);
            const float ya = ky(r - lmy), yb = ky(r - lmy - 2);
            T2 q[4] = {X::pair(xl0 + ya, xl1 + ya), X::pair(xl0 + yb, xl1 + yb), X::pair(xh0 + ya, xh1 + ya),
                       X::pair(xh0 + yb, xh1 + yb)};
            skxy[e] = *reinterpret_cast<uint4 *>(q);
        }
        __syncthreads();

        // WTA state of the lane's pixel in each patch pair: patch 2 pp + (lane >> 4), pixel lane & 15
        float best[NPP], bm1[NPP], bp1[NPP], prev[NPP], sec[B2 ? NPP : 1];
        int bd[NPP];
#pragma unroll
        for (int i = 0; i < NPP; ++i) {
            best[i] = __int_as_float(0x7f800000);
            bm1[i] = bp1[i] = prev[i] = best[i];
            if constexpr (B2) sec[i] = best[i];
            bd[i] = -1;
        }
        const float s2 = a.iscale * a.iscale;
        const T2 ns2 = X::pair(-s2, -s2);
        float *scr = escr + warp * 512;

        for (int d0 = 0; d0 < a.D; d0 += DC) {
            // ---- costs of the chunk, 16 disparities, swizzled storage
            switch (rw) {
            case 1: cost_chunk<RB, DC, 1, T, TX, TY, kThreads, 0, tc_band(RB), true>(a, sref, stgt, cbuf, vband, sstr, sstt, x0, y0, d0, tid); break;
            case 2: cost_chunk<RB, DC, 2, T, TX, TY, kThreads, 0, tc_band(RB), true>(a, sref, stgt, cbuf, vband, sstr, sstt, x0, y0, d0, tid); break;
            case 3: cost_chunk<RB, DC, 3, T, TX, TY, kThreads, 0, tc_band(RB), true>(a, sref, stgt, cbuf, vband, sstr, sstt, x0, y0, d0, tid); break;
            case 4: cost_chunk<RB, DC, 4, T, TX, TY, kThreads, 0, tc_band(RB), true>(a, sref, stgt, cbuf, vband, sstr, sstt, x0, y0, d0, tid); break;
            default: cost_chunk<RB, DC, 5, T, TX, TY, kThreads, 0, tc_band(RB), true>(a, sref, stgt, cbuf, vband, sstr, sstt, x0, y0, d0, tid); break;
            }
            // ---- aggregation, two patches at a time
#pragma unroll
            for (int pp = 0; pp < NPP; ++pp) {
                // both patches of the pair advance together, k-step by k-step
                T2 ipa[2], ipb[2];
                uint32_t brow[2];
                const T *irow[2];
                float acc[2][2][4];
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int P = warp * NPW + 2 * pp + h;
                    const int px0 = (P % NPX) * 4, py0 = (P / NPX) * 4;
                    ipa[h] = X::dup(sI[(py0 + RB + my0) * QWI + px0 + RB + mx]);
                    ipb[h] = X::dup(sI[(py0 + RB + my0 + 2) * QWI + px0 + RB + mx]);
                    const int kk = ((lane >> 3) & 1) * 8 + (lane & 7);
                    const int xq = min(px0 + kk, QW - 1);
                    const int hh = lane >> 4;
                    brow[h] = smem_addr(cbuf + ((size_t)py0 * QW + xq) * DC + ((((hh ^ (xq >> 2)) & 1)) << 3));
                    irow[h] = sI + py0 * QWI + px0 + 2 * t4;
#pragma unroll
                    for (int nb = 0; nb < 2; ++nb)
#pragma unroll
                        for (int k = 0; k < 4; ++k) acc[h][nb][k] = 0.f;
                }
#pragma unroll
                for (int r = 0; r < NKS; ++r) {
                    const uint4 kq = skxy[r * 32 + lane];
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const T2 qlo = *reinterpret_cast<const T2 *>(irow[h] + r * QWI);
                        const T2 qhi = *reinterpret_cast<const T2 *>(irow[h] + r * QWI + 8);
                        const T2 dla = __hsub2(qlo, ipa[h]), dlb = __hsub2(qlo, ipb[h]);
                        const T2 dha = __hsub2(qhi, ipa[h]), dhb = __hsub2(qhi, ipb[h]);
                        uint32_t af[4];
                        af[0] = X::ex2(__hfma2(__hmul2(dla, ns2), dla, *reinterpret_cast<const T2 *>(&kq.x)));
                        af[1] = X::ex2(__hfma2(__hmul2(dlb, ns2), dlb, *reinterpret_cast<const T2 *>(&kq.y)));
                        af[2] = X::ex2(__hfma2(__hmul2(dha, ns2), dha, *reinterpret_cast<const T2 *>(&kq.z)));
                        af[3] = X::ex2(__hfma2(__hmul2(dhb, ns2), dhb, *reinterpret_cast<const T2 *>(&kq.w)));
                        uint32_t b0, b1, b2, b3;
                        ldsm_x4_t(brow[h] + (uint32_t)(r * QW * DC * (int)sizeof(T)), b0, b1, b2, b3);
                        X::mma(acc[h][0], af, b0, b1);
                        X::mma(acc[h][1], af, b2, b3);
                    }
                }
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    float *sb = scr + h * 256;
#pragma unroll
                    for (int nb = 0; nb < 2; ++nb) {
                        const int u = 2 * nb + (t4 >> 1), o = 2 * (t4 & 1);
                        *reinterpret_cast<float2 *>(sb + g * 16 + ((u ^ tc_eswz(g)) << 2) + o) =
                            make_float2(acc[h][nb][0], acc[h][nb][1]);
                        *reinterpret_cast<float2 *>(sb + (g + 8) * 16 + ((u ^ tc_eswz(g + 8)) << 2) + o) =
                            make_float2(acc[h][nb][2], acc[h][nb][3]);
                    }
                }
                __syncwarp();
                // running WTA over the chunk, lowest d first
                {
                    const int m = lane & 15, fm = tc_eswz(m);
                    const float *er = scr + (lane >> 4) * 256 + m * 16;
                    float e[16];
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const float4 v = *reinterpret_cast<const float4 *>(er + ((u ^ fm) << 2));
                        e[4 * u] = v.x;
                        e[4 * u + 1] = v.y;
                        e[4 * u + 2] = v.z;
                        e[4 * u + 3] = v.w;
                    }
                    const int dn = min(DC, a.D - d0);
#pragma unroll
                    for (int dd = 0; dd < DC; ++dd) {
                        const int d = d0 + dd;
                        if (dn < DC && dd >= dn) break;
                        const float v = e[dd];
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
                __syncwarp();
            }
            __syncthreads();
        }

        // ---- epilogue: eq. (subpixel), add back s_i(v), validity from the row table
#pragma unroll
        for (int pp = 0; pp < NPP; ++pp) {
            const int P = warp * NPW + 2 * pp + (lane >> 4), m = lane & 15;
            const int u = x0 + (P % NPX) * 4 + (m & 3), v = y0 + (P / NPX) * 4 + (m >> 2);
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
                // the skipped normaliser sum_q w(p,q), in FP32 from the same exponent
                const int px = (P % NPX) * 4 + (m & 3), py = (P / NPX) * 4 + (m >> 2);
                const float ip = (float)sI[(py + RB) * QWI + px + RB];
                float ws = 0.f;
                for (int dx = 0; dx < KB; ++dx)
                    for (int dy = 0; dy < KB; ++dy) {
                        const float t = ((float)sI[(py + dy) * QWI + px + dx] - ip) * a.iscale;
                        ws += ex2_approx(fmaf(-t, t, a.K[dx * KB + dy]));
                    }
                a.best2[2 * o] = best[pp] / ws;
                a.best2[2 * o + 1] = sec[pp] / ws;
            }
        }
    }  // tile loop
}

template <typename T, bool B2 = false>
FusedKernel pick_tc_rb(int rb)
{
    switch (rb) {
    case 0: return k_fused_tc<0, T, B2>;
    case 1: return k_fused_tc<1, T, B2>;
    case 2: return k_fused_tc<2, T, B2>;
    case 3: return k_fused_tc<3, T, B2>;
    case 4: return k_fused_tc<4, T, B2>;
    case 5: return k_fused_tc<5, T, B2>;
    case 6: return k_fused_tc<6, T, B2>;
    }
    return nullptr;
}

}  // namespace sgb
