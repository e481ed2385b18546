// dmn_solve_warp.cu -- instances of the warp-per-point solve (solve_warp.cuh)
// for depths 6 and 7, and its host-side sizes; depth 8 is in
// dmn_solve_warp8.cu (the translation units compile in parallel).
// Thermoelastic and J2 leaves, mixed precision; four warps (four points, in
// lockstep) per CTA, register budget for 2, 3 or 4 CTAs per SM (variants 22,
// 23, 24).
#include "solve_warp.cuh"

namespace dmn {

namespace {
constexpr int kWarpsPerCta = 4;

template <int K>
KernelFn pick_k(int minb) {
  if (minb <= 2) return dmn_solve_warp<K, kWarpsPerCta, 2, 1>;
  if (minb == 3) return dmn_solve_warp<K, kWarpsPerCta, 3, 1>;
  return dmn_solve_warp<K, kWarpsPerCta, 4, 1>;
}
}  // namespace

int warp_form_warps() { return kWarpsPerCta; }

bool warp_form_supports(int K, bool mixed, int law) { return mixed && K >= 6 && K <= 8 && law == 1; }

size_t warp_smem_bytes(int K, int n_mats) {
  const size_t mp = sizeof(MatPt<float, dfl>);
  const size_t head = (n_mats * mp + 15) & ~size_t(15);
  return head + size_t(kWarpsPerCta) * size_t(warp_detail::wlay_bytes(K, n_mats, int(mp))) +
         size_t(warp_detail::up_bytes(kWarpsPerCta));
}

size_t warp_scratch_bytes_per_cta(int K) {
  return sizeof(float) * size_t(kWarpsPerCta) * size_t(warp_detail::wscratch_floats(K));
}

KernelFn warp_kernel(int K, int minb) {
  if (K == 6) return pick_k<6>(minb);
  if (K == 7) return pick_k<7>(minb);
  return warp_kernel8(minb);
}

// the index-check log of this translation unit (debug build; dmn_check.cuh)
DMN_BOUNDS_TU(bounds_log_warp)

}  // namespace dmn
