// k_fused_f32_tiles.cu -- FP32 instantiations of the fused kernel with the 32 x 72 tile that
// the batch autotuner can choose (the 128 x 18 tile is in k_fused_f32_wc4.cu; one translation
// unit each keeps the parallel build short).
#include "k_fused.cuh"

namespace sgb {

FusedKernel pick_fused_f32_tiles(int rb, int dc, int wc)
{
    if (dc != 12) return nullptr;
    if (wc == 1) return pick_rb<12, float, 1>(rb);
    if (wc == 4) return pick_fused_f32_wc4(rb);
    return nullptr;
}

}  // namespace sgb
