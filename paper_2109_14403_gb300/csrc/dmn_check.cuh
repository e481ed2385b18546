// dmn_check.cuh -- index checks of the debug build.
//
// Built with -DDMN_BOUNDS_CHECK (the library libdmn_debug.so), every node,
// leaf, state-offset and scratch index the solve kernels use goes through
// DMN_IDX(i, n): an index outside [0, n) is recorded -- the first violation's
// source line, index and bound in a device-wide log, and a flag of the
// point being evaluated -- and replaced by 0, so the access that follows
// stays inside the array.  The kernel then gives the point the status bit
// DMN_PT_BOUNDS.  Nothing traps: the launch completes and the host reads
// the log (dmn_debug_bounds_log).  In the release build DMN_IDX(i, n) is i.
#pragma once
#include <cuda_runtime.h>

namespace dmn {

constexpr int kPtBounds = 16;  // per-point status bit (DMN_PT_BOUNDS)

#ifdef DMN_BOUNDS_CHECK
struct BoundsLog {
  unsigned int count;  // violations seen
  int line, index, bound;  // the first one
};
extern __device__ BoundsLog g_bounds_log;

// the flag of the point a warp evaluates (one per warp slot of the CTA)
__device__ __forceinline__ int *bounds_flags() {
  __shared__ int flags[32];
  return flags;
}
__device__ __forceinline__ int &bounds_flag_of_point(int warp_of_point) { return bounds_flags()[warp_of_point]; }

__device__ __noinline__ void bounds_record(int line, long long i, long long n);

__device__ __forceinline__ long long checked_index(long long i, long long n, int line, int slot) {
  if (i < 0 || i >= n) {
    bounds_record(line, i, n);
    bounds_flags()[slot] = 1;
    return 0;
  }
  return i;
}
#define DMN_IDX(i, n) ((decltype(i))::dmn::checked_index((long long)(i), (long long)(n), __LINE__, \
                                                         int(threadIdx.x >> 5) & 31))
// the point-level flag: cleared when a point starts, read when it ends.
// A CTA-per-point kernel uses slot 0 for its point; a warp-per-point kernel
// the warp's slot, and every check of a CTA-per-point kernel writes its
// warp's slot too, so that kernel ORs the flags of all its warps.
#define DMN_BOUNDS_CLEAR(slot) (::dmn::bounds_flags()[(slot)] = 0)
#define DMN_BOUNDS_GET(slot) (::dmn::bounds_flags()[(slot)])
#else
#define DMN_IDX(i, n) (i)
#define DMN_BOUNDS_CLEAR(slot) ((void)0)
#define DMN_BOUNDS_GET(slot) 0
#endif

}  // namespace dmn
