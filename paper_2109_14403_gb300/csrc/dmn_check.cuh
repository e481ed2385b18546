// dmn_check.cuh -- index checks of the debug build.
//
// Built with -DDMN_BOUNDS_CHECK (the library libdmn_debug.so), every node,
// leaf, point, state-offset and shared-memory slot index the solve kernels
// use goes through DMN_IDX(i, n) (an int): an index outside [0, n) is recorded -- a
// count, and the first violation's source line, index and bound, in a log
// in device memory -- and replaced by 0, so the access that follows stays
// inside its array; the warp's flag is set, and the kernel gives the point
// it was evaluating the status bit DMN_PT_BOUNDS.  Nothing traps: the
// launch completes and the host reads the log (dmn_debug_bounds_log).
// In the release build DMN_IDX(i, n) is i and the flags do not exist.
//
// Each translation unit that includes this header keeps its own log (no
// relocatable device code is needed); those with solve kernels name a host
// accessor with DMN_BOUNDS_TU(name), which dmn_debug_bounds_log calls.
#pragma once
#include <cuda_runtime.h>

namespace dmn {

constexpr int kPtBounds = 16;  // per-point status bit (DMN_PT_BOUNDS)

struct BoundsLog {
  unsigned long long count;   // violations seen
  long long index, bound;     // the first one: index, bound
  int line, pad_;             // and its source line
};

#ifdef DMN_BOUNDS_CHECK
// internal linkage: one log per translation unit
static __device__ BoundsLog g_bounds_log;

static __device__ __noinline__ void bounds_record(int line, long long i, long long n) {
  if (atomicAdd(&g_bounds_log.count, 1ull) == 0ull) {
    g_bounds_log.index = i;
    g_bounds_log.bound = n;
    g_bounds_log.line = line;
  }
}

// one flag per warp of the CTA: the warp met a bad index during its point
__device__ __forceinline__ int *bounds_flags() {
  __shared__ int flags[32];
  return flags;
}

__device__ __forceinline__ long long checked_index(long long i, long long n, int line) {
  if (i < 0 || i >= n) {
    bounds_record(line, i, n);
    bounds_flags()[threadIdx.x >> 5] = 1;
    return 0;
  }
  return i;
}
#define DMN_IDX(i, n) (static_cast<int>(::dmn::checked_index((long long)(i), (long long)(n), __LINE__)))
// the calling warp's flag: cleared by its lane 0 when a point starts (the
// warp's present lanes then meet: a point of fewer than 32 threads is a
// partial warp), read when the point ends
#define DMN_BOUNDS_CLEAR()                                                    \
  do {                                                                        \
    const unsigned dmn_m_ = __activemask();                                   \
    if ((threadIdx.x & 31) == 0) ::dmn::bounds_flags()[threadIdx.x >> 5] = 0; \
    __syncwarp(dmn_m_);                                                       \
  } while (0)
#define DMN_BOUNDS_GET() (::dmn::bounds_flags()[threadIdx.x >> 5])
// CTA-per-point kernels: the flags of all the CTA's warps (a __syncthreads_or)
#define DMN_BOUNDS_CTA_OR() __syncthreads_or(DMN_BOUNDS_GET())
// host accessor of this translation unit's log: copy it out, optionally clear it
#define DMN_BOUNDS_TU(name)                                                      \
  cudaError_t name(BoundsLog *out, bool clear) {                                 \
    cudaError_t e = cudaMemcpyFromSymbol(out, g_bounds_log, sizeof(BoundsLog)); \
    if (e == cudaSuccess && clear) {                                             \
      const BoundsLog z = {0ull, 0ll, 0ll, 0, 0};                                \
      e = cudaMemcpyToSymbol(g_bounds_log, &z, sizeof(BoundsLog));               \
    }                                                                            \
    return e;                                                                    \
  }
#else
#define DMN_IDX(i, n) (i)
#define DMN_BOUNDS_CLEAR() ((void)0)
#define DMN_BOUNDS_GET() 0
#define DMN_BOUNDS_CTA_OR() 0
#define DMN_BOUNDS_TU(name)                                \
  cudaError_t name(BoundsLog *out, bool) {                 \
    *out = BoundsLog{0ull, 0ll, 0ll, 0, 0};                \
    return cudaErrorNotSupported;                          \
  }
#endif

}  // namespace dmn
