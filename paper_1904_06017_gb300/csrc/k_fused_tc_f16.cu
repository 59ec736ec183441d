// k_fused_tc_f16.cu -- FP16 instantiations of the tensor-core fused kernel, and the choice
// between the two storage types.
#include "k_fused_tc.cuh"

namespace sgb {

FusedKernel pick_fused_tc_bf16(int rb);

FusedKernel pick_fused_tc(int cost_dtype, int rb)
{
    if (cost_dtype == STEREO_F16) return pick_tc_rb<__half>(rb);
    if (cost_dtype == STEREO_BF16) return pick_fused_tc_bf16(rb);
    return nullptr;
}

}  // namespace sgb
