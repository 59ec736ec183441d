// k_fused_tc_bf16_b2.cu -- BF16 instantiations of the tensor-core fused kernel with the best2 output.
#include "k_fused_tc.cuh"

namespace sgb {

FusedKernel pick_fused_tc_bf16_b2(int rb) { return pick_tc_rb<__nv_bfloat16, true>(rb); }

}  // namespace sgb
