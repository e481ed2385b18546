// dmn_solve_compact_vp.cu -- instances of the compact solve (solve_compact.cuh)
// that also handle the Perzyna leaf (material kind 2), depth K <= 9.
#include "solve_compact.cuh"

namespace dmn {

KernelFn compact_kernel_vp(int K, bool mixed) {
  if (K <= 8)
    return mixed ? dmn_solve_compact<float, dfl, 128, 3, 2> : dmn_solve_compact<double, double, 128, 1, 2>;
  return mixed ? dmn_solve_compact<float, dfl, 256, 1, 2> : dmn_solve_compact<double, double, 256, 1, 2>;
}

// the index-check log of this translation unit (debug build; dmn_check.cuh)
DMN_BOUNDS_TU(bounds_log_compact_vp)

}  // namespace dmn
