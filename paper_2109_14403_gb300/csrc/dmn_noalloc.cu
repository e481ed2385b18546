// dmn_noalloc.cu -- dmn_eval_noalloc: one load increment without any device
// allocation.
//
// Who needs it: callers that may not call cudaMalloc at all -- for example a
// material routine invoked by a host finite-element code inside a region
// where the device allocator must not be touched (a memory pool owned by
// another runtime, a real-time or sandboxed plug-in), or code that cannot
// keep a handle alive between calls.  dmn_create allocates the handle's
// tables and its work-queue counter with cudaMalloc; this entry point takes
// the same tree and material description from host memory on every call and
// places everything the solve kernel needs besides the caller's inputs and
// outputs in one file-scope device array.
//
// The array is a static __device__ object: every GPU that loads the library
// holds kScratchBytes of it until the process exits.  Its host-side name is
// only a stand-in for the device object, so the device address is looked up
// once per device (cudaGetSymbolAddress, with that device current) and that
// address is what the kernel receives.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <atomic>

#include "../../include/dmn.h"
#include "dmn_internal.h"

using namespace dmn;

namespace {

constexpr int kNoAllocMaxK = 8;                 // largest supported depth
constexpr size_t kScratchBytes = 64 * 1024;     // 64 KiB per device
constexpr int kMaxDevices = 64;

// node tables, leaf tables, material table and the work-queue counter
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// device address of the array, per device (nullptr until looked up); host
// threads that make their first call on a device at the same time may both
// look it up, and both store the same address
static std::atomic<void *> g_scratch_addr[kMaxDevices];

// errors are reported through dmn_last_error() like every other call
dmn_status na_fail(dmn_status s, const char *fmt, ...) {
  char msg[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(msg, sizeof(msg), fmt, ap);
  va_end(ap);
  set_error_message(msg);
  return s;
}

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace

extern "C" dmn_status dmn_eval_noalloc(int32_t K, const double *leaf_w, const double *normals,
                                       const uint8_t *phase_map, const dmn_material *mats,
                                       int32_t n_mats, const dmn_options *opt, dmn_stream stream,
                                       int64_t n_points, const double *d_deps, const double *d_theta,
                                       double dt, const double *d_state_in, double *d_state_out,
                                       double *d_out, int32_t *d_status, int32_t *d_iters) {
  set_error_message("");
  if (K < 1 || K > kNoAllocMaxK)
    return na_fail(DMN_ERR_ARG,
                   "dmn_eval_noalloc: K=%d outside 1..%d (the static scratch array holds the "
                   "tables of trees up to depth %d)",
                   K, kNoAllocMaxK, kNoAllocMaxK);
  if (!leaf_w || !normals || !phase_map || !mats)
    return na_fail(DMN_ERR_ARG, "dmn_eval_noalloc: NULL host array argument");
  if (n_mats < 1 || n_mats > kMaxMats)
    return na_fail(DMN_ERR_ARG, "dmn_eval_noalloc: n_mats=%d outside 1..%d", n_mats, kMaxMats);
  if (n_points < 0) return na_fail(DMN_ERR_ARG, "dmn_eval_noalloc: n_points < 0");
  if (n_points == 0) return DMN_OK;
  if (!d_deps || !d_theta || !d_state_in || !d_state_out || !d_out || !d_status || !d_iters)
    return na_fail(DMN_ERR_ARG, "dmn_eval_noalloc: NULL device pointer");
  if (!(dt > 0.0) || !isfinite(dt)) return na_fail(DMN_ERR_ARG, "dmn_eval_noalloc: dt must be > 0");
  dmn_options o;
  if (opt) o = *opt; else dmn_default_options(&o);
  if (!(o.tol > 0.0) || !(o.gamma > 0.0 && o.gamma < 1.0) || o.maxit < 1 || o.maxbacktrack < 0 ||
      (o.precision != DMN_PREC_FP64 && o.precision != DMN_PREC_MIXED) ||
      !solve_variant_valid(o.solve_variant))
    return na_fail(DMN_ERR_ARG, "dmn_eval_noalloc: invalid options");
  if (is_warp_variant(o.solve_variant))
    return na_fail(DMN_ERR_ARG,
                   "dmn_eval_noalloc: solve_variant %d (one warp per point) needs the scratch of a dmn_handle",
                   o.solve_variant);

  const int nleaf = 1 << K, N = nleaf - 1;
  // ---- host tables: fixed-size arrays on the stack (no heap either).  The
  //      caller's leaf weights and phase map are copied too, so that every
  //      upload below reads call-local memory only ----
  constexpr int NMAX = (1 << kNoAllocMaxK) - 1, LMAX = 1 << kNoAllocMaxK;
  double mat[kMatWords * kMaxMats];
  double node[kNodeWords * NMAX];
  float node_df[kNodeDfl * NMAX];
  double wscr[LMAX], lw[LMAX];
  int zoff[LMAX], hoff[LMAX];
  uint8_t ph[LMAX];
  for (int j = 0; j < nleaf; ++j) {
    lw[j] = leaf_w[j];
    ph[j] = phase_map[j];
  }
  TreeLayout lay;
  char why[256];
  if (build_tree_tables(K, lw, normals, ph, mats, n_mats, mat, node, node_df, zoff, hoff, wscr, &lay,
                        why, sizeof(why)))
    return na_fail(DMN_ERR_ARG, "dmn_eval_noalloc: %s", why);
  if (lay.law == 3)
    return na_fail(DMN_ERR_ARG, "dmn_eval_noalloc: PA66 leaves (kind 3) need a dmn_handle");
  if (!(o.res_floor > 0.0)) o.res_floor = 1e-8 * lay.Emax;
  const int law = lay.law, zend = lay.zend, zw = lay.zw, SW = lay.SW;
  const size_t sbytes = sizeof(double) * (size_t)SW * (size_t)n_points;
  const char *sa = (const char *)d_state_in, *sb = (const char *)d_state_out;
  if (sa < sb + sbytes && sb < sa + sbytes)
    return na_fail(DMN_ERR_ARG, "dmn_eval_noalloc: state_in overlaps state_out");
  if ((((uintptr_t)d_state_in) & 15) || (((uintptr_t)d_state_out) & 15))
    return na_fail(DMN_ERR_ARG, "dmn_eval_noalloc: state buffers must be 16-byte aligned");

  // ---- scratch layout ----
  const size_t o_queue = 0;
  const size_t o_node = align256(o_queue + sizeof(unsigned long long));
  const size_t o_ndf = align256(o_node + sizeof(double) * kNodeWords * N);
  const size_t o_leafw = align256(o_ndf + sizeof(float) * kNodeDfl * N);
  const size_t o_phase = align256(o_leafw + sizeof(double) * nleaf);
  const size_t o_zoff = align256(o_phase + nleaf);
  const size_t o_mat = align256(o_zoff + sizeof(int) * nleaf);
  const size_t used = o_mat + sizeof(double) * kMatWords * n_mats;
  if (used > kScratchBytes)
    return na_fail(DMN_ERR_INTERNAL, "dmn_eval_noalloc: tables need %zu bytes of scratch", used);

  // ---- per-device set-up: the device address of the scratch array ----
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return na_fail(DMN_ERR_CUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return na_fail(DMN_ERR_INTERNAL, "device %d out of range", dev);
  void *addr = g_scratch_addr[dev].load(std::memory_order_acquire);
  if (!addr) {
    e = cudaGetSymbolAddress(&addr, g_noalloc_scratch);
    if (e != cudaSuccess)
      return na_fail(DMN_ERR_CUDA, "cudaGetSymbolAddress: %s", cudaGetErrorString(e));
    g_scratch_addr[dev].store(addr, std::memory_order_release);
  }
  unsigned char *base = static_cast<unsigned char *>(addr);
  const bool mixed = o.precision == DMN_PREC_MIXED;
  int num_sms = 0, smem_optin = 0, blocks_per_sm = 0;
  cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (solve_smem_bytes(K, zw, n_mats, mixed, o.solve_variant, law) > (size_t)smem_optin)
    return na_fail(DMN_ERR_ARG, "dmn_eval_noalloc: K=%d does not fit one SM in this precision", K);
  e = prepare_solve(K, zw, n_mats, mixed, o.solve_variant, law, &blocks_per_sm);
  if (e != cudaSuccess) return na_fail(DMN_ERR_CUDA, "prepare_solve: %s", cudaGetErrorString(e));
  if (blocks_per_sm < 1) return na_fail(DMN_ERR_ARG, "dmn_eval_noalloc: kernel does not fit one SM");

  // ---- upload the tables (stream-ordered copies from the call-local
  //      arrays above, which are pageable memory: the copy is staged before
  //      cudaMemcpyAsync returns, so they may go out of scope on return) ----
  cudaStream_t s = (cudaStream_t)stream;
  struct {
    size_t off;
    const void *src;
    size_t bytes;
  } up[] = {{o_node, node, sizeof(double) * kNodeWords * N},
            {o_ndf, node_df, sizeof(float) * kNodeDfl * N},
            {o_leafw, lw, sizeof(double) * nleaf},
            {o_phase, ph, (size_t)nleaf},
            {o_zoff, zoff, sizeof(int) * nleaf},
            {o_mat, mat, sizeof(double) * kMatWords * n_mats}};
  for (const auto &u : up) {
    e = cudaMemcpyAsync(base + u.off, u.src, u.bytes, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return na_fail(DMN_ERR_CUDA, "cudaMemcpyAsync: %s", cudaGetErrorString(e));
  }

  SolveParams P;
  memset(&P, 0, sizeof(P));
  P.K = K;
  P.N = N;
  P.G = 1 << (K - 1);
  P.SW = SW;
  P.zend = zend;
  P.n_mats = n_mats;
  P.maxit = o.maxit;
  P.maxbt = o.maxbacktrack;
  P.tol = o.tol;
  P.gamma = o.gamma;
  P.res_floor = o.res_floor;
  P.dt = dt;
  P.node = reinterpret_cast<const double *>(base + o_node);
  P.node_df = reinterpret_cast<const float *>(base + o_ndf);
  P.leafw = reinterpret_cast<const double *>(base + o_leafw);
  P.phase = reinterpret_cast<const uint8_t *>(base + o_phase);
  P.zoff = reinterpret_cast<const int *>(base + o_zoff);
  P.mat = reinterpret_cast<const double *>(base + o_mat);
  P.zw = zw;
  P.law = law;
  P.queue = reinterpret_cast<unsigned long long *>(base + o_queue);  // zeroed by launch_solve
  P.n_points = n_points;
  P.deps = d_deps;
  P.theta = d_theta;
  P.sin = d_state_in;
  P.sout = d_state_out;
  P.out = d_out;
  P.status = d_status;
  P.iters = d_iters;
  int64_t grid = (int64_t)num_sms * blocks_per_sm;
  if (grid > n_points) grid = n_points;
  e = launch_solve(P, mixed, o.solve_variant, (int)grid, s);
  if (e != cudaSuccess) return na_fail(DMN_ERR_CUDA, "dmn_eval_noalloc launch: %s", cudaGetErrorString(e));
  return DMN_OK;
}
