// solve_common.cuh -- device helpers shared by the two solve kernels
// (dmn_solve.cu: owner-mapped tree sweeps; dmn_solve_compact.cu: compact
// levels and incremental strains).
#pragma once
#include "dmn_kernels.cuh"

namespace dmn {

enum { ACT_STEP = 0, ACT_BACK = 1, ACT_DONE = 2 };
constexpr int kPtStaging = 32;  // per-point status bit (DMN_PT_STAGING_TIMEOUT)

template <typename TF>
struct Ctrl {
  TF res, res_old, gi, pad0_;
  unsigned long long next;  // point taken from the queue
  int action, it, bt, status, first, nonfinite;
  int lead;  // warp that runs the levels of at most 32 nodes (compact kernel)
  int pad_;
};

__device__ __forceinline__ unsigned group_mask(int G) {
  return G >= 32 ? 0xffffffffu : ((1u << G) - 1u);
}
// shuffle segment width: a point with fewer than 32 threads is one segment
__device__ __forceinline__ int group_width(int G) { return G >= 32 ? 32 : G; }

// ------------------------------------------------------------------ cache hints
// Per-point data (state blocks, predicted increments, parked internal
// variables) is read once and streamed past L1, which then keeps the node
// tables that every pass of every point reads (L1 is what shared memory
// leaves over, about 28 KB per SM at three CTAs).
__device__ __forceinline__ double ld_stream(const double *p) {
  double v;
  asm("ld.global.nc.L1::no_allocate.f64 %0, [%1];" : "=d"(v) : "l"(p));
  return v;
}
__device__ __forceinline__ float ld_stream(const float *p) {
  float v;
  asm("ld.global.nc.L1::no_allocate.f32 %0, [%1];" : "=f"(v) : "l"(p));
  return v;
}
// coherent load that does not allocate in L1 (data written earlier in the
// same launch by this CTA, read once)
template <typename T>
__device__ __forceinline__ T ld_once(const T *p) {
  static_assert(sizeof(T) == 8, "8-byte values");
  unsigned long long b;
  asm volatile("ld.global.L1::no_allocate.b64 %0, [%1];" : "=l"(b) : "l"(p) : "memory");
  T v;
  memcpy(&v, &b, 8);
  return v;
}
__device__ __forceinline__ double ld_keep(const double *p) {
  double v;
  asm("ld.global.nc.L1::evict_last.f64 %0, [%1];" : "=d"(v) : "l"(p));
  return v;
}
__device__ __forceinline__ float ld_keep(const float *p) {
  float v;
  asm("ld.global.nc.L1::evict_last.f32 %0, [%1];" : "=f"(v) : "l"(p));
  return v;
}
__device__ __forceinline__ float4 ld_keep(const float4 *p) {
  float4 v;
  asm("ld.global.nc.L1::evict_last.v4.f32 {%0, %1, %2, %3}, [%4];"
      : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
      : "l"(p));
  return v;
}

// ------------------------------------------------------------------ node constants
template <typename HP>
struct NodeHP {
  HP n[3], ns[3], c1, c2;  // normal, normal / sqrt2, volume fractions
};
__device__ __forceinline__ void load_node(const SolveParams &P, int p, NodeHP<double> &o) {
  p = DMN_IDX(p, P.N);
  const double *r = P.node + kNodeWords * p;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    o.n[i] = ld_keep(r + i);
    o.ns[i] = ld_keep(r + 8 + i);
  }
  o.c1 = ld_keep(r + 3);
  o.c2 = ld_keep(r + 4);
}
__device__ __forceinline__ void load_node(const SolveParams &P, int p, NodeHP<dfl> &o) {
  p = DMN_IDX(p, P.N);
  const float4 *r = reinterpret_cast<const float4 *>(P.node_df + kNodeDfl * p);
  const float4 a = ld_keep(r), b = ld_keep(r + 1), c = ld_keep(r + 2), d = ld_keep(r + 3);
  o.n[0] = {a.x, a.y};
  o.n[1] = {a.z, a.w};
  o.n[2] = {b.x, b.y};
  o.ns[0] = {b.z, b.w};
  o.ns[1] = {c.x, c.y};
  o.ns[2] = {c.z, c.w};
  o.c1 = {d.x, d.y};
  o.c2 = {d.z, d.w};
}
// normal, c1, c2, 1/(w c1 c2), w c1 c2 in the condensation precision
__device__ __forceinline__ void load_node_tf(const SolveParams &P, int p, double n[3], double &c1,
                                             double &c2, double &iwcc, double &wcc) {
  p = DMN_IDX(p, P.N);
  const double *r = P.node + kNodeWords * p;
  n[0] = ld_keep(r);
  n[1] = ld_keep(r + 1);
  n[2] = ld_keep(r + 2);
  c1 = ld_keep(r + 3);
  c2 = ld_keep(r + 4);
  wcc = ld_keep(r + 6);
  iwcc = ld_keep(r + 7);
}
__device__ __forceinline__ void load_node_tf(const SolveParams &P, int p, float n[3], float &c1,
                                             float &c2, float &iwcc, float &wcc) {
  p = DMN_IDX(p, P.N);
  const float *r = P.node_df + kNodeDfl * p;
  n[0] = ld_keep(r);
  n[1] = ld_keep(r + 2);
  n[2] = ld_keep(r + 4);
  c1 = ld_keep(r + 12);
  c2 = ld_keep(r + 14);
  iwcc = ld_keep(r + 16);
  wcc = ld_keep(r + 17);
}

// B a = sym(a (x) n) with the pre-scaled normal ns = n / sqrt2
template <typename HP>
__device__ __forceinline__ void bvec_hp(const NodeHP<HP> &nd, const HP a[3], HP out[6]) {
  out[0] = a[0] * nd.n[0];
  out[1] = a[1] * nd.n[1];
  out[2] = a[2] * nd.n[2];
  out[3] = a[1] * nd.ns[2] + a[2] * nd.ns[1];
  out[4] = a[0] * nd.ns[2] + a[2] * nd.ns[0];
  out[5] = a[0] * nd.ns[1] + a[1] * nd.ns[0];
}

// B^T s = s n (traction) in HP; the cancellation of the residual happens
// here, so it must run in the high precision before any rounding to TF
template <typename HP>
__device__ __forceinline__ void btvec_hp(const NodeHP<HP> &nd, const HP s[6], HP out[3]) {
  out[0] = s[0] * nd.n[0] + s[5] * nd.ns[1] + s[4] * nd.ns[2];
  out[1] = s[1] * nd.n[1] + s[5] * nd.ns[0] + s[3] * nd.ns[2];
  out[2] = s[2] * nd.n[2] + s[4] * nd.ns[0] + s[3] * nd.ns[1];
}

// Debug build: a leaf's phase row, and the offsets of its internal variables
// in shared memory (hq: their copy, or the PA66 history) and in the state
// block (zq, from the end of the jumps), inside their arrays; violations are
// recorded and replaced by 0 (dmn_check.cuh).  The release build leaves the
// values as they are.
template <typename M>
__device__ __forceinline__ void check_leaf(const SolveParams &P, const M *mp, int &ph, int &hq, int &zq,
                                           int ZW) {
#ifdef DMN_BOUNDS_CHECK
  ph = DMN_IDX(ph, P.n_mats);
  const int kind = mp[ph].kind;
  if (zq >= 0) {
    const int nh = kind == 3 ? kPaHist : (kind == 2 ? 13 : 7);
    const int nz = kind == 3 ? kPaZ : (kind == 2 ? 13 : 7);
    hq = DMN_IDX(hq, ZW - nh + 1);
    zq = DMN_IDX(zq, P.zend - (8 + 3 * P.N) - nz + 1);
  }
#else
  (void)P, (void)mp, (void)ph, (void)hq, (void)zq, (void)ZW;
#endif
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v, unsigned mask, int W) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1)
    if (o < W) v = v + hp_shfl_down(mask, v, o, W);
  return v;
}

}  // namespace dmn
