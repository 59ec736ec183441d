// k_fused_sc16.cu -- the FP16 / BF16 storage form on the screened kernel's tensor-core
// aggregation (tile code kScWC): a running WTA on the 16-bit sums, no refinement.
#include "k_fused_sc.cuh"

namespace sgb {

FusedKernel pick_fused_sc16(int cost_dtype, int rb)
{
    if (rb > kScMaxRB) return nullptr;
    if (cost_dtype == STEREO_F16) return pick_sc_rb<false, kScPlain, __half>(rb);
    if (cost_dtype == STEREO_BF16) return pick_sc_rb<false, kScPlain, __nv_bfloat16>(rb);
    return nullptr;
}

}  // namespace sgb
