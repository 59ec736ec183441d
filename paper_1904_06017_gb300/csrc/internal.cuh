// internal.cuh -- declarations shared by the translation units of the library.
// Not part of the C ABI (include/stereo.h is).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "stereo.h"

namespace sgb {

// Tiling of the fused kernel: a CTA of kWarps warps owns a tile of output pixels; lane =
// column, each warp covers 32 columns x kPY rows, and WC warp columns x (kWarps / WC) warp rows
// give tiles of 32 x 72 (WC = 1), 64 x 36 (WC = 2, the default) or 128 x 18 (WC = 4).
constexpr int kPY = 6;
constexpr int kWarps = 12;
constexpr int kThreads = 32 * kWarps;
constexpr int kDefaultWC = 2;
// The warp-specialised form (tile code kWsWC): 8 producer warps compute the costs of the next
// chunk while 8 consumer warps aggregate the current one, on 64 x 16 tiles (2 consumer warp
// columns x 4 consumer warp rows x kWsPY pixels per thread).
constexpr int kWsWC = 8;
constexpr int kWsProdWarps = 8;
constexpr int kWsConsWarps = 8;
constexpr int kWsThreads = 32 * (kWsProdWarps + kWsConsWarps);
constexpr int kWsPY = 4;
constexpr int kWsBand = 3;          // cost rows per band of the producers' two-pass window sums
constexpr int kWsMaxRB = 5;         // the two cost buffers fit shared memory up to bil = 11
// The tensor-core form (tile code kTcWC, FP16 / BF16 storage): 64 x 36 tiles, kWarps warps,
// 16 disparities per chunk, aggregation by mma.sync over 4 x 4 pixel patches, bil <= 13.
constexpr int kTcWC = 16;
constexpr int kTcMaxRB = 6;
constexpr float kTcMaxSigma1 = 150.f;   // -s^2 stays a normal FP16 number
// The screened FP32 form (tile code kScWC): 32 x 36 tiles, kWarps warps, tensor-core screening
// over 32 disparities per chunk and an exact FP32 refinement of the certified candidates
// (k_fused_sc.cuh); bil <= 13 (at 13 a window row fills the 16 k-slots of an mma).
constexpr int kScWC = 32;
constexpr int kScMaxRB = 6;
__host__ __device__ constexpr int tile_x(int wc)
{
    return wc == kWsWC || wc == kTcWC ? 64 : wc == kScWC ? 32 : 32 * wc;
}
__host__ __device__ constexpr int tile_y(int wc)
{
    return wc == kWsWC ? kWsPY * (kWsConsWarps / 2) : wc == kTcWC || wc == kScWC ? 36 : kPY * (kWarps / wc);
}
// Whether the tensor-core form can run these parameters.
inline bool tc_supported(int cost_dtype, int bil, float sigma1)
{
    return cost_dtype != STEREO_F32 && bil / 2 <= kTcMaxRB && sigma1 <= kTcMaxSigma1;
}
__host__ __device__ constexpr int fused_threads(int wc) { return wc == kWsWC ? kWsThreads : kThreads; }
constexpr int kMaxRB = 7;          // bil <= 15
constexpr int kMaxRW = 5;          // win <= 11
constexpr int kMaxD = 256;
constexpr int kMaxDim = 16384;
constexpr int kProfSlots = 4096;
constexpr int kDtThreads = 256;
constexpr int kDtMaxBlocks = 1024;   // partial-moment blocks of the disparity transformation

// Derived geometry of a context (all sizes in pixels / bytes).
struct Geometry {
    int W, H, pitch, D, rw, rb, m, n;
    int dc;            // disparities per chunk of the fused kernel
    int wc;            // warp columns of a fused-kernel tile (tile_x(wc) x tile_y(wc) pixels)
    int tx, ty;        // tile size
    int esize;         // bytes per stored cost (4 for FP32, 2 for FP16 / BF16)
    int Dp;            // D rounded up to a multiple of dc
    int ntx, nty;      // tiles
    int pad_left, pad_top, pad_w, pad_h, pad_pitch;   // replicate-padded staging images
    int ref_box_w, tgt_box_w, box_h;                  // TMA boxes (bytes x rows)
    int ref_e, tgt_e;  // column offset of image column x0 - m (resp. x0 - m - (Dp-1)) in the box
    size_t smem_bytes; // dynamic shared memory of the fused kernel
};

}  // namespace sgb

struct stereo_ctx {
    stereo_params p;
    sgb::Geometry g;
    int device;
    int nsm;                       // SMs of the device (grid of the persistent screened kernel)
    uint8_t *ref_pad, *tgt_pad;    // replicate-padded copies (pad_pitch x pad_h)
    int2 *ref_stats, *tgt_stats;   // per padded position: {sum, bits of 1/sqrt(n*sumsq - sum^2)}
    int4 *row_tab;                 // per image row: {s_i(v), max and min of s_i over rows v-m..v+m,
                                   //   min over those rows of the target's column-0 run length}
    CUtensorMap tmap_ref, tmap_tgt;
    float kspatial[(2 * sgb::kMaxRB + 1) * (2 * sgb::kMaxRB + 1)];  // -log2(e) |dq|^2 / sigma0^2
    float iscale;                  // sqrt(log2(e)) / sigma1
    double *mom_part;              // [kDtMaxBlocks][10] partial moments
    float *dt_coef;                // 3 FP32 coefficients of the final per-pixel map
    stereo_dt_result *res_dev;     // device-side result when the caller passes none
    int *status_dev;               // device status word (bounded waits)
    int stall_test;                // test hook of stereo_debug_stall_staging
    // LR-consistency check (stereo_create only; batch contexts leave them null)
    uint8_t *lr_ref, *lr_tgt;      // mirrored warped target and mirrored reference [H][pitch]
    int32_t *lr_wta;               // target-view WTA of the mirrored pair [H][W]
    float *lr_disp;                // the mirrored run's disparity output (unused) [H][W]
    // fused-kernel timing
    int prof_on;
    int prof_n;
    std::vector<cudaEvent_t> prof_ev;
};

namespace sgb {

int set_error(int code, const char *fmt, ...);
int cuda_error(cudaError_t e, const char *what);

// Launchers (each returns STEREO_OK or an error code; they only enqueue work).
int launch_warp(stereo_ctx *ctx, const uint8_t *tgt, const float *shift, uint8_t *out,
                cudaStream_t s);
int launch_prep(stereo_ctx *ctx, const uint8_t *ref, const uint8_t *tgtw, cudaStream_t s);
int launch_row_tables(stereo_ctx *ctx, const float *shift, const uint8_t *tgtw, cudaStream_t s);
int launch_fused(stereo_ctx *ctx, const float *shift, float *disp, int32_t *wta, uint8_t *valid,
                 cudaStream_t s, float *best2 = nullptr);
size_t fused_smem_bytes(const Geometry &g);
int fused_configure(stereo_ctx *ctx);
int compute_geometry(const stereo_params &p, int dc, int wc, Geometry &g);
// Context creation with a given (disparities per chunk, warp columns); 0 = default choice.
int create_context(const stereo_params *p, int dc, int wc, stereo_ctx **out);
int max_smem_optin();
int launch_cost_volume(stereo_ctx *ctx, float *cost, cudaStream_t s);
int launch_aggregate_volume(stereo_ctx *ctx, const uint8_t *ref, const float *cost, float *agg,
                            cudaStream_t s);
int launch_wta_volume(stereo_ctx *ctx, const float *agg, const float *shift, float *disp,
                      int32_t *wta, float *best2, cudaStream_t s);
int launch_dt(stereo_ctx *ctx, const float *disp, const uint8_t *mask, double psi_init,
              float delta_t, float *out, stereo_dt_result *res_dev, cudaStream_t s);
int run_fp32_probe(int blocks_per_sm, double *gflops_scalar, double *gflops_packed);

// Kernels of the disparity transformation (k_dt.cu), shared with its no-allocation entry point.
int dt_moment_blocks(size_t n_pixels);   // blocks of k_dt_moments for a map of n_pixels
__global__ void k_dt_moments(const float *__restrict__ disp, const uint8_t *__restrict__ mask, int W, int H,
                             double *__restrict__ part);
__global__ void k_dt_solve(const double *__restrict__ part, int nblocks, int W, int H, double psi_init,
                           double lambda0, double delta_psi, int max_iters, float delta_t,
                           stereo_dt_result *__restrict__ res, float *__restrict__ coef);
__global__ void k_dt_apply(const float *__restrict__ disp, int W, int H, const float *__restrict__ coef,
                           float *__restrict__ out);

}  // namespace sgb
