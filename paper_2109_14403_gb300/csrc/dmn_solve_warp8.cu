// dmn_solve_warp8.cu -- depth-8 instances of the warp-per-point solve
// (solve_warp.cuh): four warps per CTA, register budget for 2, 3 or 4 CTAs
// per SM.
#include "solve_warp.cuh"

namespace dmn {

KernelFn warp_kernel8(int minb) {
  if (minb <= 2) return dmn_solve_warp<8, 4, 2, 1>;
  if (minb == 3) return dmn_solve_warp<8, 4, 3, 1>;
  return dmn_solve_warp<8, 4, 4, 1>;
}

// the index-check log of this translation unit (debug build; dmn_check.cuh)
DMN_BOUNDS_TU(bounds_log_warp8)

}  // namespace dmn
