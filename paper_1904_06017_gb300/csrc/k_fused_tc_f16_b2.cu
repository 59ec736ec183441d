// k_fused_tc_f16_b2.cu -- FP16 instantiations of the tensor-core fused kernel with the best2
// output, and the choice between the two storage types.
#include "k_fused_tc.cuh"

namespace sgb {

FusedKernel pick_fused_tc_bf16_b2(int rb);

FusedKernel pick_fused_tc_b2(int cost_dtype, int rb)
{
    if (cost_dtype == STEREO_F16) return pick_tc_rb<__half, true>(rb);
    if (cost_dtype == STEREO_BF16) return pick_fused_tc_bf16_b2(rb);
    return nullptr;
}

}  // namespace sgb
