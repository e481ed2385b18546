// dmn_solve_compact.cu -- instances of the compact solve (solve_compact.cuh)
// for thermoelastic and J2 leaves, depth K <= 8, and its shared-memory size.
#include "solve_compact.cuh"

namespace dmn {

size_t compact_smem_bytes(int K, int zw, int n_mats, bool mixed) {
  const int N = (1 << K) - 1, G = 1 << (K - 1);
  const size_t hp = 8, tf = mixed ? 4 : 8;
  const Scratch sc = scratch_layout(G, int(tf));
  size_t b = hp * (3 * N + 6 * G + zw + 18 + 6 + 4 + sc.words);
  b += (mixed ? sizeof(MatPt<float, dfl>) : sizeof(MatPt<double, double>)) * n_mats;
  b = (b + 15) & ~size_t(15);
  b += mixed ? sizeof(Ctrl<float>) : sizeof(Ctrl<double>);
  b += tf * (32 + 40 + 24 * N);
  return (b + 15) & ~size_t(15);
}

KernelFn compact_kernel(int K, bool mixed, int minb) {
  (void)K;  // depth <= 8: at most 128 threads
  if (!mixed) return dmn_solve_compact<double, double, 128, 1, 1>;
  if (minb >= 4) return dmn_solve_compact<float, dfl, 128, 4, 1>;
  return minb == 3 ? dmn_solve_compact<float, dfl, 128, 3, 1> : dmn_solve_compact<float, dfl, 128, 2, 1>;
}

// the index-check log of this translation unit (debug build; dmn_check.cuh)
DMN_BOUNDS_TU(bounds_log_compact)

}  // namespace dmn
