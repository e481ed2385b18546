// dmn_solve_compact_pa66.cu -- instances of the compact solve (solve_compact.cuh)
// that also handle the PA66 leaf (material kind 3, pa66.cuh), depth K <= 8,
// and their shared-memory size.
#include "solve_compact.cuh"

namespace dmn {

size_t compact_smem_bytes_pa(int K, int hw, int n_mats, bool mixed) {
  const size_t pa = mixed ? sizeof(MatPA<float, dfl>) : sizeof(MatPA<double, double>);
  return compact_smem_bytes(K, hw, n_mats, mixed) + pa * n_mats + 16;
}

KernelFn compact_kernel_pa66(int K, bool mixed) {
  (void)K;  // depth <= 8: at most 128 threads
  return mixed ? dmn_solve_compact<float, dfl, 128, 2, 3> : dmn_solve_compact<double, double, 128, 1, 3>;
}

// the index-check log of this translation unit (debug build; dmn_check.cuh)
DMN_BOUNDS_TU(bounds_log_compact_pa66)

}  // namespace dmn
