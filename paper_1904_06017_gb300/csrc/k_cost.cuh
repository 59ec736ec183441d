// k_cost.cuh -- the cost phase of the fused kernels: eq. (c) for one chunk of disparities at a
// tile plus its bilateral halo, into shared memory.  Two forms:
//   cost_chunk      -- vertical running sums of the products per (product column, d) and
//                      horizontal sums over the w columns, band by band of cost rows;
//   cost_chunk_mma  -- the cross term on the tensor cores (exact FP16 operands and FP32
//                      accumulation), one warp per block of 8 cost columns.
#pragma once
#include <type_traits>

#include "k_fused_common.cuh"

namespace sgb {

// One cost rounded to the storage type.
template <typename T> __device__ __forceinline__ T cost_from_float(float c);
template <> __device__ __forceinline__ float cost_from_float<float>(float c) { return c; }
template <> __device__ __forceinline__ __half cost_from_float<__half>(float c) { return __float2half_rn(c); }
template <> __device__ __forceinline__ __nv_bfloat16 cost_from_float<__nv_bfloat16>(float c)
{
    return __float2bfloat16_rn(c);
}

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
template <int BAR, int NT>
__device__ __forceinline__ void group_sync()
{
    if constexpr (BAR == 0) __syncthreads();
    else asm volatile("bar.sync %0, %1;" ::"n"(BAR), "n"(NT) : "memory");
}

// SWZ: the DC disparities of a position are stored as DC / 8 16-byte units whose index is XORed
// with a function of the column (the tensor-core aggregations' ldmatrix layouts): for DC = 16
// unit ^ bit 2 of the column, for DC = 32 unit ^ bits 1..2 of the column (sc_unit below).
// CSH: the costs are stored multiplied by 2^CSH (exactly: the power of two is folded into the
// reciprocal and the constant of eq. (c), so the scaled value is the same rounding of the same
// exact product).  PLW > 0: planar storage, one plane per disparity, rows of PLW entries and
// planes PSZ entries apart (cbuf[d * PSZ + y * PLW + x]), for per-pixel gathers whose lanes need
// different disparities; with PAIR the planes hold disparity pairs (2k, 2k + 1) interleaved as
// float2, cbuf[(k * PSZ + y * PLW + x) * 2 + (d & 1)], so that one 8-byte load gives both.
// KSEG: cost columns per work item of the horizontal pass.
template <int DC>
__host__ __device__ constexpr int swz_unit(int unit, int x)
{
    return DC == 16 ? unit ^ ((x >> 2) & 1) : unit ^ ((x >> 1) & 3);
}

template <int RB, int DC, int RW, typename T, int TX, int TY, int NT = kThreads, int BAR = 0,
          int KBAND = kBand, bool SWZ = false, int CSH = 0, int PLW = 0, int PSZ = 0, int KSEG = kSeg,
          bool PAIR = false>
__device__ __forceinline__ void cost_chunk(const FusedArgs &a, const uint8_t *sref, const uint8_t *stgt,
                                           T *cbuf, int *vband, int2 *sstr, int2 *sstt,
                                           int x0, int y0, int d0, int tid)
{
    constexpr int kThreads = NT, kBand = KBAND, kSeg = KSEG;   // the threads, band and segment of this instantiation
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
        constexpr int kSub = kBand <= 6 ? kBand : kBand % 6 == 0 ? 6 : kBand % 8 == 0 ? 8 : kBand % 4 == 0 ? 4 : 1;
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
            constexpr float CS = (float)(1 << CSH);
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
                const float ir = __int_as_float(rs[j].y) * CS;
                const int2 t0 = ts[j + 3], t1 = ts[j + 2], t2 = ts[j + 1], t3 = ts[j];
                out[j].x = fmaf(-(float)(a.n * S.x - rs[j].x * t0.x), ir * __int_as_float(t0.y), CS);
                out[j].y = fmaf(-(float)(a.n * S.y - rs[j].x * t1.x), ir * __int_as_float(t1.y), CS);
                out[j].z = fmaf(-(float)(a.n * S.z - rs[j].x * t2.x), ir * __int_as_float(t2.y), CS);
                out[j].w = fmaf(-(float)(a.n * S.w - rs[j].x * t3.x), ir * __int_as_float(t3.y), CS);
                if (j + 1 < kSeg) {
                    S.x += v[j + WS].x - v[j].x;
                    S.y += v[j + WS].y - v[j].y;
                    S.z += v[j + WS].z - v[j].z;
                    S.w += v[j + WS].w - v[j].w;
                }
            }
            if constexpr (SWZ) {
                // DC / 8 16-byte units per position, the unit index swizzled by the column
                static_assert(DC == 16 || DC == 32, "swizzled layouts hold 16 or 32 disparities per position");
                T *co = cbuf + (size_t)yq * crow + 4 * (dq & 1);
#pragma unroll
                for (int j = 0; j < kSeg; ++j) {
                    const int x = xs + j;
                    if (j < nout) CostStore<T>::store4(co + (size_t)x * DC + (swz_unit<DC>(dq >> 1, x) << 3), out[j]);
                }
            } else if constexpr (PLW > 0 && PAIR) {
                static_assert(PSZ >= QH * PLW, "planes must not overlap");
                static_assert(std::is_same<T, float>::value, "pair planes hold FP32 costs");
                float2 *co = reinterpret_cast<float2 *>(cbuf) + (size_t)(2 * dq) * PSZ + (size_t)yq * PLW;
#pragma unroll
                for (int j = 0; j < kSeg; ++j)
                    if (j < nout) {
                        const int x = xs + j;
                        co[x] = make_float2(out[j].x, out[j].y);
                        co[PSZ + x] = make_float2(out[j].z, out[j].w);
                    }
            } else if constexpr (PLW > 0) {
                static_assert(PSZ >= QH * PLW, "planes must not overlap");
                T *co = cbuf + (size_t)(4 * dq) * PSZ + (size_t)yq * PLW;
#pragma unroll
                for (int j = 0; j < kSeg; ++j)
                    if (j < nout) {
                        const int x = xs + j;
                        co[x] = cost_from_float<T>(out[j].x);
                        co[PSZ + x] = cost_from_float<T>(out[j].y);
                        co[2 * PSZ + x] = cost_from_float<T>(out[j].z);
                        co[3 * PSZ + x] = cost_from_float<T>(out[j].w);
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

}  // namespace sgb
