// k_fused_bf16.cu -- BF16 cost storage instantiations of the fused kernel.
#include "k_fused.cuh"

namespace sgb {

FusedKernel pick_fused_bf16(int rb, int dc, int wc)
{
    if (dc == 12 && wc == 2) return pick_rb<12, __nv_bfloat16, 2>(rb);
    return nullptr;
}

}  // namespace sgb
