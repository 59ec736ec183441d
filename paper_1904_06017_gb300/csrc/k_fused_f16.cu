// k_fused_f16.cu -- FP16 cost storage instantiations of the fused kernel.
#include "k_fused.cuh"

namespace sgb {

FusedKernel pick_fused_f16(int rb, int dc, int wc)
{
    if (dc == 12 && wc == 2) return pick_rb<12, __half, 2>(rb);
    return nullptr;
}

}  // namespace sgb
