// k_fused_b2_f32.cu -- FP32 instantiations of the fused kernel with the best2 output (the
// smallest E over d != d* tracked beside the running WTA), for single-pair contexts (WC = 2,
// 12 disparities per chunk); and the choice of a best2 kernel for a context.
#include "k_fused.cuh"
#include "k_fused_tc.cuh"

namespace sgb {

FusedKernel pick_fused_f32_b2(int rb, int dc)
{
    if (dc == 12) return pick_rb<12, float, 2, true>(rb);
    return nullptr;
}

FusedKernel pick_fused_b2(int cost_dtype, int rb, int dc, int wc)
{
    if (wc == kTcWC) return dc == kTcDC && rb <= kTcMaxRB ? pick_fused_tc_b2(cost_dtype, rb) : nullptr;
    if (wc == kScWC) return cost_dtype == STEREO_F32 ? pick_fused_sc_b2(rb) : pick_fused_sc16_b2(cost_dtype, rb);
    if (cost_dtype == STEREO_F32 && wc == 2) return pick_fused_f32_b2(rb, dc);
    return nullptr;
}

}  // namespace sgb
