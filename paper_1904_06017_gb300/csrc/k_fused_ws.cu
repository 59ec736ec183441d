// k_fused_ws.cu -- instantiations of the warp-specialised fused kernel (FP32 cost storage,
// 12 disparities per chunk, bilateral radius up to kWsMaxRB).
#include "k_fused_ws.cuh"

namespace sgb {

FusedKernel pick_fused_ws(int rb, int dc)
{
    if (dc != 12) return nullptr;
    switch (rb) {
    case 0: return k_fused_ws<0, 12, float>;
    case 1: return k_fused_ws<1, 12, float>;
    case 2: return k_fused_ws<2, 12, float>;
    case 3: return k_fused_ws<3, 12, float>;
    case 4: return k_fused_ws<4, 12, float>;
    case 5: return k_fused_ws<5, 12, float>;
    }
    return nullptr;
}

}  // namespace sgb
