// k_fused_sc_b2.cu -- the screened FP32 fused kernel with the best2 output: every pixel refines
// all D disparities in FP32, so the smallest E over d != d* is k_fused's value too.
#include "k_fused_sc.cuh"

namespace sgb {

FusedKernel pick_fused_sc_b2(int rb) { return rb <= kScMaxRB ? pick_sc_rb<true>(rb) : nullptr; }

}  // namespace sgb
