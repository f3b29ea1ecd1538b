// Instances of the persistent inner iteration (loop_kernels.cuh), one per
// register-prefetch warp-apply shape and pointwise item size, in a
// translation unit of their own so that they compile beside the engine.
#include "engine.h"
#include "loop_kernels.cuh"

namespace heat {

template <int SX, int NY, int W, int MINB>
static LoopFn loop_for(int qpt) {
  // FP32_REFINED instance: the FP32 paths differ only in the inner
  // iteration cap, which update_item takes from the simulation
  switch (qpt) {
    case 1: return k_cg_loop<P_FP32_REFINED, SX, NY, W, MINB, 1, E_Q1>;
    case 2: return k_cg_loop<P_FP32_REFINED, SX, NY, W, MINB, 2, E_Q1>;
    case 4: return k_cg_loop<P_FP32_REFINED, SX, NY, W, MINB, 4, E_Q1>;
    default: return nullptr;
  }
}

LoopFn loop_kernel(int sx, int ny, int warps, int qpt) {
  if (sx == 16 && ny == 4 && warps == 4) return loop_for<16, 4, 4, 3>(qpt);
  if (sx == 32 && ny == 4 && warps == 4) return loop_for<32, 4, 4, 3>(qpt);
  if (sx == 16 && ny == 2 && warps == 8) return loop_for<16, 2, 8, 2>(qpt);
  if (sx == 32 && ny == 2 && warps == 4) return loop_for<32, 2, 4, 4>(qpt);
  return nullptr;
}

}  // namespace heat
