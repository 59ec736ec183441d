// k_fused_f32.cu -- FP32 cost storage instantiations of the fused kernel, and the host
// side shared by all storage types (shared-memory sizing, kernel choice, launch).
#include <string.h>

#include <algorithm>

#include "k_fused.cuh"
#include "k_fused_sc.cuh"

namespace sgb {

FusedKernel pick_fused_f32(int rb, int dc, int wc)
{
    if (wc != 2) return pick_fused_f32_tiles(rb, dc, wc);
    if (dc == 12) return pick_rb<12, float, 2>(rb);
    if (dc == 4) return pick_fused_f32_dc4(rb);
    return nullptr;
}

FusedKernel pick_fused(int cost_dtype, int rb, int dc, int wc)
{
    if (wc == kWsWC) return cost_dtype == STEREO_F32 && rb <= kWsMaxRB ? pick_fused_ws(rb, dc) : nullptr;
    if (wc == kTcWC) return dc == kTcDC && rb <= kTcMaxRB ? pick_fused_tc(cost_dtype, rb) : nullptr;
    if (wc == kScWC) {
        if (dc != kScDC) return nullptr;
        return cost_dtype == STEREO_F32 ? pick_fused_sc(rb) : pick_fused_sc16(cost_dtype, rb);
    }
    switch (cost_dtype) {
    case STEREO_F32: return pick_fused_f32(rb, dc, wc);
    case STEREO_F16: return pick_fused_f16(rb, dc, wc);
    case STEREO_BF16: return pick_fused_bf16(rb, dc, wc);
    }
    return nullptr;
}

size_t fused_smem_bytes(const Geometry &g)
{
    if (g.wc == kTcWC) return tc_layout(g.rb, g.m, g.ref_box_w, g.tgt_box_w, g.box_h, g.esize).total;
    if (g.wc == kScWC) return sc_layout(g.rb, g.m, g.ref_box_w, g.tgt_box_w, g.box_h).total;
    // the warp-specialised form keeps the two-pass cost phase (vband, staged statistics); the
    // others compute costs on the tensor cores and need neither
    const bool ws = g.wc == kWsWC;
    return smem_layout(g.rb, g.m, g.dc, g.ref_box_w, g.tgt_box_w, g.box_h, g.esize, g.tx, g.ty, ws ? 2 : 1,
                       ws ? kWsBand : 0)
        .total;
}

static FusedKernel pick(const stereo_ctx *ctx)
{
    return pick_fused(ctx->p.cost_dtype, ctx->g.rb, ctx->g.dc, ctx->g.wc);
}

int fused_configure(stereo_ctx *ctx)
{
    FusedKernel k = pick(ctx);
    if (!k)
        return set_error(STEREO_ENOTSUP, "no fused kernel for bil=%d dc=%d cost_dtype=%d", ctx->p.bil, ctx->g.dc,
                         ctx->p.cost_dtype);
    int rc = cuda_error(cudaFuncSetAttribute((const void *)k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)ctx->g.smem_bytes),
                        "cudaFuncSetAttribute(fused)");
    FusedKernel k2 = pick_fused_b2(ctx->p.cost_dtype, ctx->g.rb, ctx->g.dc, ctx->g.wc);
    if (!rc && k2)
        rc = cuda_error(cudaFuncSetAttribute((const void *)k2, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)ctx->g.smem_bytes),
                        "cudaFuncSetAttribute(fused, best2)");
    return rc;
}

// The pair descriptor of a context for one call (outputs are per call).
void fill_pair_desc(const stereo_ctx *ctx, float *disp, int32_t *wta, uint8_t *valid, PairDesc &d, float *best2)
{
    const Geometry &g = ctx->g;
    FusedArgs &a = d.a;
    memset(&d, 0, sizeof(d));
    d.tmap_ref = ctx->tmap_ref;
    d.tmap_tgt = ctx->tmap_tgt;
    d.ntx = g.ntx;
    d.nty = g.nty;
    a.ref_stats = ctx->ref_stats;
    a.tgt_stats = ctx->tgt_stats;
    a.row_tab = ctx->row_tab;
    a.disp = disp;
    a.wta = wta;
    a.valid = valid;
    a.best2 = best2;
    a.status = ctx->status_dev;
    a.stall_test = ctx->stall_test;
    a.W = g.W;
    a.H = g.H;
    a.D = g.D;
    a.Dp = g.Dp;
    a.rw = g.rw;
    a.m = g.m;
    a.n = g.n;
    a.pad_left = g.pad_left;
    a.pad_top = g.pad_top;
    a.pad_w = g.pad_w;
    a.ref_e = g.ref_e;
    a.tgt_e = g.tgt_e;
    a.ref_box_w = g.ref_box_w;
    a.tgt_box_w = g.tgt_box_w;
    a.box_h = g.box_h;
    a.ref_box_x = g.pad_left - (int)align_up(g.m, 16);
    a.iscale = ctx->iscale;
    const int kb = 2 * g.rb + 1;
    for (int i = 0; i < kb * kb; ++i) a.K[i] = ctx->kspatial[i];
}

int launch_fused(stereo_ctx *ctx, const float *shift, float *disp, int32_t *wta, uint8_t *valid,
                 cudaStream_t s, float *best2)
{
    (void)shift;   // the integer shifts come from the row table built by k_row_tables
    const Geometry &g = ctx->g;
    FusedKernel k = best2 ? pick_fused_b2(ctx->p.cost_dtype, g.rb, g.dc, g.wc) : pick(ctx);
    if (!k)
        return set_error(STEREO_ENOTSUP, best2 ? "the best2 output needs FP32 storage (the screened form or 12 "
                                                 "disparities per chunk) or the tensor-core form (FP16 / BF16 with bil <= 13)"
                                               : "no fused kernel for bil=%d",
                         ctx->p.bil);
    PairDesc d;
    fill_pair_desc(ctx, disp, wta, valid, d, best2);
    const int ntiles = g.ntx * g.nty;
    // the screened form is persistent (one CTA per SM, tiles in turn, the next tile's images
    // staged while the current one finishes); the others take one tile per CTA
    const int grid = g.wc == kScWC ? std::min(ntiles, ctx->nsm) : ntiles;
    k<<<grid, fused_threads(g.wc), g.smem_bytes, s>>>(d, nullptr, nullptr, ntiles, nullptr);
    return cuda_error(cudaGetLastError(), "k_fused launch");
}

}  // namespace sgb
