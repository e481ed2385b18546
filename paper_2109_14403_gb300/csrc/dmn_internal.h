// dmn_internal.h -- declarations shared by the library's translation units.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>

#include "dmn_kernels.cuh"

namespace dmn {
// shared memory of the selected solve kernel (variant as in dmn_options)
size_t solve_smem_bytes(int K, int nz, int n_mats, bool mixed, int variant);
bool solve_variant_valid(int variant);
// the compact solve kernel (dmn_solve_compact.cu), depth K <= 8
using KernelFn = void (*)(const SolveParams);
size_t compact_smem_bytes(int K, int nz, int n_mats, bool mixed);
KernelFn compact_kernel(int K, bool mixed, int minb);
cudaError_t prepare_solve(int K, int nz, int n_mats, bool mixed, int variant, int *blocks_per_sm);
cudaError_t launch_solve(const SolveParams &P, bool mixed, int variant, int grid, cudaStream_t s);
// message returned by dmn_last_error() on this thread
void set_error_message(const char *msg);
}  // namespace dmn
