// dmn_internal.h -- declarations shared by the library's translation units.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>

#include "../../include/dmn.h"
#include "dmn_kernels.cuh"

namespace dmn {
// shared memory of the selected solve kernel (variant as in dmn_options; law:
// largest material kind of the tree, 1 or 2; zw: internal-variable words)
size_t solve_smem_bytes(int K, int zw, int n_mats, bool mixed, int variant, int law);
bool solve_variant_valid(int variant);
// the compact solve kernel: dmn_solve_compact.cu (kinds 0 and 1, K <= 8) and
// dmn_solve_compact_vp.cu (also kind 2, K <= 9)
using KernelFn = void (*)(const SolveParams);
size_t compact_smem_bytes(int K, int zw, int n_mats, bool mixed);
KernelFn compact_kernel(int K, bool mixed, int minb);
KernelFn compact_kernel_vp(int K, bool mixed);
// ... and dmn_solve_compact_pa66.cu (also kind 3, K <= 8; hw: history words)
size_t compact_smem_bytes_pa(int K, int hw, int n_mats, bool mixed);
KernelFn compact_kernel_pa66(int K, bool mixed);
// host: validate a material and write its device row (kMatWords doubles);
// returns nullptr or the reason it is invalid
const char *material_row(const dmn_material &m, double row[kMatWords]);
// words of internal variables of a leaf of this kind (0, 7, 13 or 79), and
// the words of shared memory the solve keeps for it (kind 3: its history)
int material_z_words(int kind);
int material_hist_words(int kind);
// Tree setup of Sec. 3.1 on the host, into caller-provided arrays (so that a
// caller without a heap can use it): validates the materials, leaf weights
// (> 0, sum 1), phase map and normals; writes the material rows
// mat[n_mats][kMatWords], the node tables node[N][kNodeWords] and
// node_df[N][kNodeDfl] (weight propagation bottom-up, normalised normals),
// the state offsets zoff[2^K] of the leaves' internal variables and, with
// PA66 leaves, the shared-memory offsets hoff[2^K] of their history.
// wscratch: 2^K doubles.  Returns nullptr, or the reason the input is invalid.
struct TreeLayout {
  int SW, zend, zw, law, hw;  // state words, end of z, z words, largest kind, history words
  double Emax;                // largest Young's modulus (default residual floor)
};
const char *build_tree_tables(int K, const double *leaf_w, const double *normals,
                              const uint8_t *phase_map, const dmn_material *mats, int n_mats,
                              double *mat, double *node, float *node_df, int *zoff, int *hoff,
                              double *wscratch, TreeLayout *lay, char *why, size_t why_len);
// the warp-per-point form (dmn_solve_warp.cu, dmn_solve_warp8.cu): variants
// 22..24 (CTAs per SM the register budget is sized for: variant - 20), depth
// 6..8, kinds 0 and 1, mixed precision; it needs a scratch slot per resident
// warp
bool is_warp_variant(int variant);
bool warp_form_supports(int K, bool mixed, int law);
int warp_form_warps();
size_t warp_smem_bytes(int K, int n_mats);
size_t warp_scratch_bytes_per_cta(int K);
KernelFn warp_kernel(int K, int minb);
KernelFn warp_kernel8(int minb);
// threads per CTA of the kernel a variant selects
int solve_block_threads(int K, int variant, int law);
cudaError_t prepare_solve(int K, int zw, int n_mats, bool mixed, int variant, int law,
                          int *blocks_per_sm);
cudaError_t launch_solve(const SolveParams &P, bool mixed, int variant, int grid, cudaStream_t s);
// dmn_eval_mixed (dmn_drive.cu): prescribed strain components, outer = 0 and
// optionally the tangent predictor; one outer Newton update after an
// evaluation; the status bit of the points given up
cudaError_t mixed_prepare(cudaStream_t s, int64_t n, int sw, const uint8_t *mask,
                          const double *target, double *deps, double *theta, double dt,
                          double c_heat, const double *sin, const double *out, bool predict,
                          int32_t *outer);
cudaError_t mixed_update(cudaStream_t s, int64_t n, int sw, int n3, const uint8_t *mask,
                         const double *target, double *deps, double *theta, double dt, double c_heat,
                         double tol, const double *sin, const double *sout, const double *out,
                         const int32_t *status, int32_t *outer, int it, bool last, float *work,
                         unsigned long long *open);
cudaError_t mixed_finish(cudaStream_t s, int64_t n, int32_t *status, int32_t *outer);
// debug build: the index-check logs of the translation units with solve
// kernels (dmn_check.cuh); cudaErrorNotSupported in the release build
cudaError_t bounds_log_owner(BoundsLog *out, bool clear);
cudaError_t bounds_log_compact(BoundsLog *out, bool clear);
cudaError_t bounds_log_compact_vp(BoundsLog *out, bool clear);
cudaError_t bounds_log_compact_pa66(BoundsLog *out, bool clear);
cudaError_t bounds_log_warp(BoundsLog *out, bool clear);
cudaError_t bounds_log_warp8(BoundsLog *out, bool clear);
// message returned by dmn_last_error() on this thread
void set_error_message(const char *msg);
}  // namespace dmn
