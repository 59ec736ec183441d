// k_fused_tc_bf16.cu -- BF16 instantiations of the tensor-core fused kernel.
#include "k_fused_tc.cuh"

namespace sgb {

FusedKernel pick_fused_tc_bf16(int rb) { return pick_tc_rb<__nv_bfloat16>(rb); }

}  // namespace sgb
