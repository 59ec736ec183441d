// k_fused_f32_dc4.cu -- FP32 instantiations of the fused kernel with 4 disparities per chunk,
// the fallback when the 12-disparity cost tile does not fit shared memory (large windows).
#include "k_fused.cuh"

namespace sgb {

FusedKernel pick_fused_f32_dc4(int rb) { return pick_rb<4, float, 2>(rb); }

}  // namespace sgb
