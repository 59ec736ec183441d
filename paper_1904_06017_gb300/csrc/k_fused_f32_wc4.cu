// k_fused_f32_wc4.cu -- FP32 instantiations of the fused kernel with 128 x 18 tiles.
#include "k_fused.cuh"

namespace sgb {

FusedKernel pick_fused_f32_wc4(int rb) { return pick_rb<12, float, 4>(rb); }

}  // namespace sgb
