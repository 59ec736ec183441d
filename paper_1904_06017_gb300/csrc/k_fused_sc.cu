// k_fused_sc.cu -- instantiations of the screened FP32 fused kernel (tile code kScWC).
#include "k_fused_sc.cuh"

namespace sgb {

FusedKernel pick_fused_sc(int rb) { return rb <= kScMaxRB ? pick_sc_rb<false>(rb) : nullptr; }

}  // namespace sgb
