// k_fused_sc16_b2.cu -- the FP16 / BF16 storage form of tile code kScWC with the best2 output.
#include "k_fused_sc.cuh"

namespace sgb {

FusedKernel pick_fused_sc16_b2(int cost_dtype, int rb)
{
    if (rb > kScMaxRB) return nullptr;
    if (cost_dtype == STEREO_F16) return pick_sc_rb<true, kScPlain, __half>(rb);
    if (cost_dtype == STEREO_BF16) return pick_sc_rb<true, kScPlain, __nv_bfloat16>(rb);
    return nullptr;
}

}  // namespace sgb
