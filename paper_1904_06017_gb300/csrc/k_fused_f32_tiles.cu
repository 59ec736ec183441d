// k_fused_f32_tiles.cu -- FP32 instantiations of the fused kernel with the other tile
// shapes (32 x 64 and 128 x 16 pixels) that the batch autotuner can choose.
#include "k_fused.cuh"

namespace sgb {

FusedKernel pick_fused_f32_tiles(int rb, int dc, int wc)
{
    if (dc != 12) return nullptr;
    if (wc == 1) return pick_rb<12, float, 1>(rb);
    if (wc == 4) return pick_rb<12, float, 4>(rb);
    return nullptr;
}

}  // namespace sgb
