// solve_common.cuh -- device helpers shared by the two solve kernels
// (dmn_solve.cu: owner-mapped tree sweeps; dmn_solve_compact.cu: compact
// levels and incremental strains).
#pragma once
#include "dmn_kernels.cuh"

namespace dmn {

enum { ACT_STEP = 0, ACT_BACK = 1, ACT_DONE = 2 };

template <typename TF>
struct Ctrl {
  TF res, res_old, gi, pad0_;
  unsigned long long next;  // point taken from the queue
  int action, it, bt, status, first, nonfinite, pad_[2];
};

__device__ __forceinline__ unsigned group_mask(int G) {
  return G >= 32 ? 0xffffffffu : ((1u << G) - 1u);
}
// shuffle segment width: a point with fewer than 32 threads is one segment
__device__ __forceinline__ int group_width(int G) { return G >= 32 ? 32 : G; }

// ------------------------------------------------------------------ node constants
template <typename HP>
struct NodeHP {
  HP n[3], ns[3], c1, c2;  // normal, normal / sqrt2, volume fractions
};
__device__ __forceinline__ void load_node(const SolveParams &P, int p, NodeHP<double> &o) {
  const double *r = P.node + kNodeWords * p;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    o.n[i] = __ldg(r + i);
    o.ns[i] = __ldg(r + 8 + i);
  }
  o.c1 = __ldg(r + 3);
  o.c2 = __ldg(r + 4);
}
__device__ __forceinline__ void load_node(const SolveParams &P, int p, NodeHP<dfl> &o) {
  const float4 *r = reinterpret_cast<const float4 *>(P.node_df + kNodeDfl * p);
  const float4 a = __ldg(r), b = __ldg(r + 1), c = __ldg(r + 2), d = __ldg(r + 3);
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
  const double *r = P.node + kNodeWords * p;
  n[0] = __ldg(r);
  n[1] = __ldg(r + 1);
  n[2] = __ldg(r + 2);
  c1 = __ldg(r + 3);
  c2 = __ldg(r + 4);
  wcc = __ldg(r + 6);
  iwcc = __ldg(r + 7);
}
__device__ __forceinline__ void load_node_tf(const SolveParams &P, int p, float n[3], float &c1,
                                             float &c2, float &iwcc, float &wcc) {
  const float *r = P.node_df + kNodeDfl * p;
  n[0] = __ldg(r);
  n[1] = __ldg(r + 2);
  n[2] = __ldg(r + 4);
  c1 = __ldg(r + 12);
  c2 = __ldg(r + 14);
  iwcc = __ldg(r + 16);
  wcc = __ldg(r + 17);
}
__device__ __forceinline__ double hp_add_tf(double a, double d) { return a + d; }
__device__ __forceinline__ dfl hp_add_tf(dfl a, float d) { return a + dfl{d, 0.0f}; }

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

template <typename T>
__device__ __forceinline__ T warp_sum(T v, unsigned mask, int W) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1)
    if (o < W) v = v + hp_shfl_down(mask, v, o, W);
  return v;
}

}  // namespace dmn
