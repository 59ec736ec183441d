// k_prep.cu -- the perspective warp of the target image (§3.1), the staging kernel that
// builds replicate-padded copies and per-position window statistics for the fused
// kernel, and an FP32 FMA throughput probe.
#include "internal.cuh"
#include "row_shift.cuh"

namespace sgb {

// §3.1: tgt_warped(u, v) = tgt(clamp(u - s_i(v), 0, W-1), v), s_i = floor(s + 0.5).
// One thread writes 16 consecutive bytes of an output row.  Where the 16 source bytes lie
// inside the row they come from the two aligned 16-byte words that cover them (rows are
// [H][pitch] with pitch a multiple of 16, so the second word ends inside the row's pitch);
// near the row ends and for unaligned buffers the bytes are read one by one.
__global__ void k_warp(const uint8_t *__restrict__ tgt, const float *__restrict__ shift,
                       uint8_t *__restrict__ out, int W, int H, int pitch)
{
    const int v = blockIdx.y;
    const int u0 = (blockIdx.x * blockDim.x + threadIdx.x) * 16;
    if (v >= H || u0 >= W) return;
    const int si = (int)round_half_up(shift[v]);
    const uint8_t *row = tgt + (size_t)v * pitch;
    uint8_t *orow = out + (size_t)v * pitch;
    const int a = u0 - si;
    const bool aligned = (((uintptr_t)tgt | (uintptr_t)out) & 15) == 0;
    if (aligned && u0 + 16 <= W && a >= 0 && a + 16 <= W) {
        const int ab = a & ~15, sh = a & 15;
        const uint4 lo = __ldg(reinterpret_cast<const uint4 *>(row + ab));
        uint4 hi = lo;
        if (sh) hi = __ldg(reinterpret_cast<const uint4 *>(row + ab + 16));
        const uint32_t w[8] = {lo.x, lo.y, lo.z, lo.w, hi.x, hi.y, hi.z, hi.w};
        const int q = sh >> 2, b = 8 * (sh & 3);
        uint32_t t[5];
#pragma unroll
        for (int k = 0; k < 5; ++k)   // the words from q on, selected without local memory
            t[k] = q == 0 ? w[k] : q == 1 ? w[k + 1] : q == 2 ? w[k + 2] : w[k + 3];
        uint32_t o[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) o[k] = __funnelshift_r(t[k], t[k + 1], b);   // bytes sh + 4k ..
        *reinterpret_cast<uint4 *>(orow + u0) = make_uint4(o[0], o[1], o[2], o[3]);
        return;
    }
    if (aligned && u0 + 16 <= W) {
        uint32_t w[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            uint32_t x = 0;
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                int src = min(max(a + 4 * k + b, 0), W - 1);
                x |= (uint32_t)__ldg(row + src) << (8 * b);
            }
            w[k] = x;
        }
        *reinterpret_cast<uint4 *>(orow + u0) = make_uint4(w[0], w[1], w[2], w[3]);
        return;
    }
    for (int u = u0; u < min(u0 + 16, W); ++u) orow[u] = __ldg(row + min(max(u - si, 0), W - 1));
}

int launch_warp(stereo_ctx *ctx, const uint8_t *tgt, const float *shift, uint8_t *out, cudaStream_t s)
{
    const Geometry &g = ctx->g;
    const int chunks = (g.W + 15) / 16;
    dim3 block(128), grid((chunks + 127) / 128, g.H);
    k_warp<<<grid, block, 0, s>>>(tgt, shift, out, g.W, g.H, g.pitch);
    return cuda_error(cudaGetLastError(), "k_warp launch");
}

// Staging: for every position (x, y) of the padded frame (image column x - pad_left,
// row y - pad_top, reads clamped to the image) write the pixel to the padded copy and
// the window statistics of the w x w block centred there:
//     {S = sum I, bits of r = 1/sqrt(n * sum I^2 - S^2)}, r = 0 for a flat block.
// These are the mu / sigma of eq. (c), kept as exact integer sums (§4.3 precomputes
// mu and sigma in global memory as well).  A block covers 32 x 32 positions: the images
// are staged with the block's halo, the horizontal window sums (sum I, sum I^2, both
// images) of every staged row are formed as running sums over groups of 4 columns, and
// each thread then walks 4 consecutive rows of one column with running vertical sums.
constexpr int kPrepX = 32, kPrepY = 8, kPrepRows = 32;   // threads x, y; positions per block in y
constexpr int kPrepG = 4;                                 // columns per horizontal running-sum item

__global__ void __launch_bounds__(kPrepX *kPrepY)
k_prep(const uint8_t *__restrict__ ref, const uint8_t *__restrict__ tgt, int W, int H, int pitch,
       int rw, int pad_left, int pad_top, int pad_w, int pad_h, int pad_pitch,
       uint8_t *__restrict__ ref_pad, uint8_t *__restrict__ tgt_pad,
       int2 *__restrict__ ref_stats, int2 *__restrict__ tgt_stats)
{
    constexpr int SX = kPrepX + 2 * kMaxRW, SY = kPrepRows + 2 * kMaxRW;
    constexpr int NT = kPrepX * kPrepY;
    __shared__ uint8_t sr[SY][SX], st[SY][SX];
    // rows padded to kPrepX + 1 words: the horizontal pass stores 4 rows x 8 column groups per
    // warp, which an unpadded stride of 32 words would put 4 to a bank
    __shared__ int hs[2][SY][kPrepX + 1], hq[2][SY][kPrepX + 1];
    const int x0 = blockIdx.x * kPrepX, y0 = blockIdx.y * kPrepRows;
    const int tid = threadIdx.y * kPrepX + threadIdx.x;
    const int ws = 2 * rw + 1;
    const int sx = kPrepX + 2 * rw, sy = kPrepRows + 2 * rw;
    for (int i = tid; i < sx * sy; i += NT) {
        const int ly = i / sx, lx = i - ly * sx;
        const int ix = min(max(x0 - rw + lx - pad_left, 0), W - 1);
        const int iy = min(max(y0 - rw + ly - pad_top, 0), H - 1);
        sr[ly][lx] = ref[(size_t)iy * pitch + ix];
        st[ly][lx] = tgt[(size_t)iy * pitch + ix];
    }
    __syncthreads();
    // horizontal sums over w columns: item = (staged row, group of kPrepG output columns),
    // the window slid across the group
    constexpr int NG = kPrepX / kPrepG;
    for (int it = tid; it < sy * NG; it += NT) {
        const int ly = it / NG, lx0 = (it - ly * NG) * kPrepG;
        int a = 0, aa = 0, b = 0, bb = 0;
        for (int j = 0; j < ws; ++j) {
            const int r = sr[ly][lx0 + j], t = st[ly][lx0 + j];
            a += r;
            aa += r * r;
            b += t;
            bb += t * t;
        }
#pragma unroll
        for (int g = 0; g < kPrepG; ++g) {
            hs[0][ly][lx0 + g] = a;
            hq[0][ly][lx0 + g] = aa;
            hs[1][ly][lx0 + g] = b;
            hq[1][ly][lx0 + g] = bb;
            if (g + 1 < kPrepG) {
                const int ro = sr[ly][lx0 + g], ri = sr[ly][lx0 + g + ws];
                const int to = st[ly][lx0 + g], ti = st[ly][lx0 + g + ws];
                a += ri - ro;
                aa += ri * ri - ro * ro;
                b += ti - to;
                bb += ti * ti - to * to;
            }
        }
    }
    __syncthreads();
    // vertical sums: this thread's column, rows ry0 .. ry0 + 3 of the block
    const int n = ws * ws;
    const int lx = threadIdx.x, ry0 = threadIdx.y * (kPrepRows / kPrepY);
    const int x = x0 + lx;
    int S[2] = {0, 0}, Q[2] = {0, 0};
    for (int j = 0; j < ws; ++j)
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            S[k] += hs[k][ry0 + j][lx];
            Q[k] += hq[k][ry0 + j][lx];
        }
    int2 *dst[2] = {ref_stats, tgt_stats};
#pragma unroll
    for (int i = 0; i < kPrepRows / kPrepY; ++i) {
        const int ly = ry0 + i, y = y0 + ly;
        if (i > 0)
#pragma unroll
            for (int k = 0; k < 2; ++k) {
                S[k] += hs[k][ly + ws - 1][lx] - hs[k][ly - 1][lx];
                Q[k] += hq[k][ly + ws - 1][lx] - hq[k][ly - 1][lx];
            }
        if (x >= pad_w || y >= pad_h) continue;
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            const int A = n * Q[k] - S[k] * S[k];   // n^2 sigma^2, exact (< 2^31 for w <= 11)
            const float r = A > 0 ? 1.0f / sqrtf((float)A) : 0.0f;
            dst[k][(size_t)y * pad_w + x] = make_int2(S[k], __float_as_int(r));
        }
        ref_pad[(size_t)y * pad_pitch + x] = sr[ly + rw][lx + rw];
        tgt_pad[(size_t)y * pad_pitch + x] = st[ly + rw][lx + rw];
    }
}

int launch_prep(stereo_ctx *ctx, const uint8_t *ref, const uint8_t *tgtw, cudaStream_t s)
{
    const Geometry &g = ctx->g;
    if (((uintptr_t)ref | (uintptr_t)tgtw) % 16)
        return set_error(STEREO_EINVAL, "images must be 16-byte aligned");
    dim3 block(kPrepX, kPrepY), grid((g.pad_w + kPrepX - 1) / kPrepX, (g.pad_h + kPrepRows - 1) / kPrepRows);
    k_prep<<<grid, block, 0, s>>>(ref, tgtw, g.W, g.H, g.pitch, g.rw, g.pad_left, g.pad_top, g.pad_w,
                                  g.pad_h, g.pad_pitch, ctx->ref_pad, ctx->tgt_pad, ctx->ref_stats,
                                  ctx->tgt_stats);
    return cuda_error(cudaGetLastError(), "k_prep launch");
}

// Per image row v: the integer shift s_i(v) = floor(s(v) + 0.5) of §3.1, the largest and
// smallest s_i over rows v-m..v+m (the validity test of the fused epilogue), and the smallest
// over those rows of L(y), the length of the run of target row y that equals its column 0 (at
// least 1; W when the whole row is one value).  The replicate padding extends that run to the
// left, so a read of row y at any column below L(y) returns the value of column 0: the
// screened fused form uses this to find the disparities beyond which every cost behind a
// pixel no longer changes.  A block of kRowTab rows first rounds its rows and an m-row halo on
// each side once and measures their runs (each warp a set of rows, 256 columns per step, the
// first step of all of them loaded together), then takes the window extremes from shared
// memory.
constexpr int kRowTab = 32, kRowTabHalo = 16;   // m = rw + bilateral radius <= 12
constexpr int kRowThreads = 256;

__global__ void __launch_bounds__(kRowThreads) k_row_tables(const float *__restrict__ shift, const uint8_t *__restrict__ tgt,
                                                           int pitch, int W, int H, int m, int4 *__restrict__ tab)
{
    __shared__ int si[kRowTab + 2 * kRowTabHalo];
    __shared__ int li[kRowTab + 2 * kRowTabHalo];
    const int v0 = blockIdx.x * kRowTab;
    for (int i = threadIdx.x; i < kRowTab + 2 * m; i += kRowThreads) {
        const int y = v0 - m + i;
        si[i] = (y >= 0 && y < H) ? (int)round_half_up(__ldg(shift + y)) : 0;
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    constexpr int kWarpsR = kRowThreads / 32, kRowsPerWarp = (kRowTab + 2 * kRowTabHalo) / kWarpsR;
    static_assert((kRowTab + 2 * kRowTabHalo) % kWarpsR == 0, "rows split evenly over the warps");
    // 256 columns of a row per step, 8 per lane (8-byte loads where the rows allow them); the
    // first step of every row of the warp is loaded up front, so that their loads are in flight
    // together, and a row that holds one value over it continues step by step
    const bool al8 = ((reinterpret_cast<uintptr_t>(tgt) | (uintptr_t)pitch) & 7) == 0;
    uint2 first[kRowsPerWarp];
    int c0v[kRowsPerWarp];
#pragma unroll
    for (int k = 0; k < kRowsPerWarp; ++k) {
        const int i = wid + k * kWarpsR, y = v0 - m + i;
        first[k] = make_uint2(0u, 0u);
        c0v[k] = 0;
        if (i < kRowTab + 2 * m && y >= 0 && y < H) {
            const uint8_t *row = tgt + (size_t)y * pitch;
            c0v[k] = __ldg(row);
            if (al8 && 8 * lane + 8 <= W) first[k] = __ldg(reinterpret_cast<const uint2 *>(row + 8 * lane));
        }
    }
#pragma unroll
    for (int k = 0; k < kRowsPerWarp; ++k) {
        const int i = wid + k * kWarpsR, y = v0 - m + i;   // warp-uniform
        if (i >= kRowTab + 2 * m) break;
        int run = 1;
        if (y >= 0 && y < H) {
            const uint8_t *row = tgt + (size_t)y * pitch;
            const int c0 = c0v[k];
            run = W;
            for (int c = 0; c < W; c += 256) {
                const int x = c + 8 * lane;
                int off = 8;   // the lane's first column (of 8) that differs from column 0
                if (al8 && x + 8 <= W) {
                    const uint2 q = c == 0 ? first[k] : __ldg(reinterpret_cast<const uint2 *>(row + x));
#pragma unroll
                    for (int j = 7; j >= 0; --j)
                        if ((int)(((j < 4 ? q.x : q.y) >> (8 * (j & 3))) & 0xffu) != c0) off = j;
                } else {
                    for (int j = 7; j >= 0; --j)
                        if (x + j < W && (int)__ldg(row + x + j) != c0) off = j;
                }
                const unsigned bm = __ballot_sync(0xffffffffu, off < 8);
                if (bm) {
                    const int src = __ffs(bm) - 1;
                    run = c + 8 * src + __shfl_sync(0xffffffffu, off, src);
                    break;
                }
            }
        }
        if (lane == 0) li[i] = run;
    }
    __syncthreads();
    const int v = v0 + threadIdx.x;
    if (threadIdx.x >= kRowTab || v >= H) return;
    int hi = -(1 << 30), lo = 1 << 30, lmin = 1 << 30;
    const int ylo = max(v - m, 0), yhi = min(v + m, H - 1);
    for (int y = ylo; y <= yhi; ++y) {
        const int s = si[y - v0 + m];
        hi = max(hi, s);
        lo = min(lo, s);
        lmin = min(lmin, li[y - v0 + m]);
    }
    tab[v] = make_int4(si[threadIdx.x + m], hi, lo, lmin);
}

int launch_row_tables(stereo_ctx *ctx, const float *shift, const uint8_t *tgtw, cudaStream_t s)
{
    const Geometry &g = ctx->g;
    if (g.m > kRowTabHalo) return set_error(STEREO_EINVAL, "k_row_tables: halo %d above %d", g.m, kRowTabHalo);
    k_row_tables<<<(g.H + kRowTab - 1) / kRowTab, kRowThreads, 0, s>>>(shift, tgtw, g.pitch, g.W, g.H, g.m, ctx->row_tab);
    return cuda_error(cudaGetLastError(), "k_row_tables launch");
}

// ------------------------------------------------------------------ FP32 probe
constexpr int kProbeChains = 8;

__global__ void __launch_bounds__(256) k_probe_scalar(float *out, int iters, float m)
{
    float acc[kProbeChains];
#pragma unroll
    for (int j = 0; j < kProbeChains; ++j) acc[j] = threadIdx.x * 1e-3f + j;
    for (int i = 0; i < iters; ++i)
#pragma unroll
        for (int j = 0; j < kProbeChains; ++j) acc[j] = fmaf(acc[j], m, 1e-3f);
    float s = 0.f;
#pragma unroll
    for (int j = 0; j < kProbeChains; ++j) s += acc[j];
    if (s == 1234.5f) out[0] = s;
}

__global__ void __launch_bounds__(256) k_probe_packed(float *out, int iters, float m)
{
    float2 acc[kProbeChains];
#pragma unroll
    for (int j = 0; j < kProbeChains; ++j) acc[j] = make_float2(threadIdx.x * 1e-3f + j, j - 1.f);
    const float2 mm = make_float2(m, m), cc = make_float2(1e-3f, 1e-3f);
    for (int i = 0; i < iters; ++i)
#pragma unroll
        for (int j = 0; j < kProbeChains; ++j) acc[j] = __ffma2_rn(acc[j], mm, cc);
    float s = 0.f;
#pragma unroll
    for (int j = 0; j < kProbeChains; ++j) s += acc[j].x + acc[j].y;
    if (s == 1234.5f) out[0] = s;
}

int run_fp32_probe(int blocks_per_sm, double *gs, double *gp)
{
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    float *out = nullptr;
    int rc = cuda_error(cudaMalloc(&out, sizeof(float)), "probe alloc");
    if (rc) return rc;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const int iters = 1 << 16, blocks = sms * blocks_per_sm;
    double res[2] = {0, 0};
    for (int kind = 0; kind < 2; ++kind) {
        float best = 1e30f;
        for (int rep = 0; rep < 4; ++rep) {
            cudaEventRecord(e0, 0);
            if (kind == 0) k_probe_scalar<<<blocks, 256>>>(out, iters, 0.999f);
            else k_probe_packed<<<blocks, 256>>>(out, iters, 0.999f);
            cudaEventRecord(e1, 0);
            cudaEventSynchronize(e1);
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (rep > 0 && ms < best) best = ms;
        }
        double fma_lanes = (double)blocks * 256 * iters * kProbeChains * (kind == 0 ? 1 : 2);
        res[kind] = 2.0 * fma_lanes / (best * 1e-3) * 1e-9;
    }
    rc = cuda_error(cudaGetLastError(), "probe kernels");
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    *gs = res[0];
    *gp = res[1];
    return rc;
}

}  // namespace sgb
