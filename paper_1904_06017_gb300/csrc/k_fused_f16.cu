// k_fused_f16.cu -- FP16 cost storage instantiations of the fused kernel.
#include "k_fused.cuh"

namespace sgb {

FusedKernel pick_fused_f16(int rb, int dc)
{
    if (dc == 12) return pick_rb<12, __half>(rb);
    return nullptr;
}

}  // namespace sgb
