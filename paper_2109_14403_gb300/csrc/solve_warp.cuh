// solve_warp.cuh -- third form of the Algorithm 1 solve (arXiv 2109.14403,
// Sec. 3.3): one warp per Gauss point, for trees of depth 6 <= K <= 8.
//
// Mapping.  Level 6 of the tree has 32 nodes: lane l owns the subtree under
// level-6 node l, i.e. M = 2^(K-6) bottom laminates (2M leaves) and the
// 2M - 1 laminates of levels 6..K above them.  A Newton pass condenses that
// subtree in the lane's registers (a postorder loop over the lane's bottom
// laminates), then the five levels 5..1 by shuffles (level k node j on lane
// j 2^(6-k)).  The loops keep one copy of the leaf, laminate and combine
// code, small enough for the instruction cache.  A CTA holds W points, one
// per warp, whose passes run in lockstep: level 5 by lane pairs on every
// warp, levels 4..1 of all W points batched on one warp (dmn_solve_warp).
//
// Strains.  Lane l keeps the strain of its level-6 node (float-float) in
// shared memory; the strains below it are formed in every pass from the
// jumps a of the lane's own nodes (eq. DMN kinematics: child 1 gets
// +c2 B a_p, child 2 -c1 B a_p).  After a Newton step the level-6 strain
// takes the float-float sum of the B da terms of its five upper ancestors,
// which the back-substitution forms on the way down anyway.
//
// Back-substitution.  da_p = -(G_p de_p + h_p) with G_p, h_p of the pass's
// condensation: for the five upper levels in shared memory, for the lane's
// own 2M - 1 nodes in a per-warp slot of global scratch memory laid out
// [node of the lane][21][lane] (a warp's stores and loads of one component
// are one 128-byte line; the slot is reused point after point, so it stays
// in L2).
//
// The condensation, the residual and the leaf laws are those of
// dmn_kernels.cuh (leaf_eval, combine), as in the other two forms.
#pragma once
#include "dmn_internal.h"
#include "solve_common.cuh"

namespace dmn {

namespace warp_detail {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kUpNodes = 31;  // levels 5..1

// per-warp shared memory, in bytes (8-byte HP, 4-byte TF), for depth K
__host__ __device__ constexpr int wlay_a(int) { return 0; }                                   // HP[3N]
__host__ __device__ constexpr int wlay_e6(int K) { return 8 * 3 * ((1 << K) - 1); }           // HP[32][6]
__host__ __device__ constexpr int wlay_trn(int K) { return wlay_e6(K) + 8 * 32 * 6; }          // HP[2^K]
__host__ __device__ constexpr int wlay_eb(int K) { return wlay_trn(K) + 8 * (1 << K); }        // HP[12], double[6]
__host__ __device__ constexpr int wlay_out(int K) { return wlay_eb(K) + 8 * 18; }              // HP[8] (sigma, D, X), TF[40]
__host__ __device__ constexpr int wlay_da(int K) { return wlay_out(K) + 8 * 8 + 4 * 40; }      // TF[3N]
__host__ __device__ constexpr int wlay_ghu(int K) { return wlay_da(K) + 4 * 3 * ((1 << K) - 1); }  // TF[31][21]
__host__ __device__ constexpr int wlay_mat(int K) {
  return (wlay_ghu(K) + 4 * kUpNodes * 21 + 15) & ~15;  // MatPt[n_mats] of the warp's point
}
// bytes of one warp's region (MatPt rows included)
__host__ __device__ inline int wlay_bytes(int K, int n_mats, int matpt_bytes) {
  return (wlay_mat(K) + n_mats * matpt_bytes + 15) & ~15;
}
// global scratch floats per warp: the lane's own 2M - 1 nodes x 21 x 32 lanes
__host__ __device__ constexpr int wscratch_floats(int K) { return (2 * (1 << (K - 6)) - 1) * 21 * 32; }

// Per-warp context of one pass
template <typename TF, typename HP>
struct WCtx {
  const SolveParams *P;
  HP *a_s;            // jumps (HP), paper node order
  TF *da_s;           // Newton increment
  const HP *trn_s;    // traces of the leaf strains at t^n
  const MatPt<TF, HP> *mp;
  float *ghw;         // the warp's global scratch slot
  const double *sin;  // the point's state block (z^n)
  double *sout;       // the point's output state block (z of the pass parked here)
  int lane;
  bool full;
  TF r2;
  HP Dsum, Xsum;
};

// node p's TF constants and HP constants
template <typename TF, typename HP>
__device__ __forceinline__ void node_all(const SolveParams &P, int p, NodeHP<HP> &nd, TF n[3], TF &c1,
                                         TF &c2, TF &iwcc, TF &wcc) {
  load_node(P, p, nd);
  load_node_tf(P, p, n, c1, c2, iwcc, wcc);
}

// children's strains of node p with strain e: e + c2 B a_p, e - c1 B a_p
template <typename HP>
__device__ __forceinline__ void child_strains(const NodeHP<HP> &nd, const HP *a, const HP e[6], HP el[6],
                                              HP er[6]) {
  const HP av[3] = {a[0], a[1], a[2]};
  HP J[6];
  bvec_hp(nd, av, J);
#pragma unroll
  for (int c = 0; c < 6; ++c) {
    el[c] = e[c] + nd.c2 * J[c];
    er[c] = e[c] - nd.c1 * J[c];
  }
}

// one leaf: its z^n from the input state (FP64 -> HP), the leaf law, its z
// of this pass parked in the output state
template <typename TF, typename HP, int LAW>
__device__ __forceinline__ void leaf_at(WCtx<TF, HP> &c, int j, const HP e[6], HP sig[6], HP &D, HP &X,
                                        Rec<TF> &rec) {
  const SolveParams &P = *c.P;
  j = DMN_IDX(j, 1 << P.K);
  const int ph = DMN_IDX(int(__ldg(P.phase + j)), P.n_mats);
  int zo = __ldg(P.zoff + j);
  const MatPt<TF, HP> &m = c.mp[ph];
  HP zn[LAW >= 2 ? 13 : 7];
  HP *znew = nullptr;
  HP *tag = nullptr;
  if (zo >= 0) {
    const int nz = (LAW >= 2 && m.kind == 2) ? 13 : 7;
    zo = DMN_IDX(zo, P.zend - nz + 1);
#pragma unroll
    for (int q = 0; q < (LAW >= 2 ? 13 : 7); ++q)
      zn[q] = q < nz ? hp_load(ld_stream(c.sin + zo + q), tag) : hp_zero(tag);
    znew = reinterpret_cast<HP *>(c.sout + zo);
  } else {
#pragma unroll
    for (int q = 0; q < (LAW >= 2 ? 13 : 7); ++q) zn[q] = hp_zero(tag);
  }
  HP zdummy[13];
  leaf_eval<TF, HP, LAW>(m, e, zn, c.trn_s[j], sig, D, X, rec, znew ? znew : zdummy, c.full);
}

// Combine the condensed records of two sibling subtrees (L: child 1, in/out;
// R: child 2) into node p's record, with the residual of p from the
// children's plain stress sums (S_L in/out becomes S_L + S_R); G/h of p into
// gh.  The same code serves the lane's own levels and the shuffle levels.
template <typename TF, typename HP>
__device__ __forceinline__ void combine_node(const SolveParams &P, int p, Rec<TF> &L, const Rec<TF> &R, HP SL[6],
                                             const HP SR[6], TF &r2, bool full, TF *gh) {
  NodeHP<HP> nd;
  load_node(P, p, nd);
  HP dh[6];
#pragma unroll
  for (int q = 0; q < 6; ++q) {
    dh[q] = nd.c2 * SL[q] - nd.c1 * SR[q];
    SL[q] = SL[q] + SR[q];
  }
  HP rh[3];
  btvec_hp(nd, dh, rh);  // r_p = B^T (c2 S_L - c1 S_R)
  TF n[3], c1, c2, iwcc, wcc;
  load_node_tf(P, p, n, c1, c2, iwcc, wcc);
  TF rv[3];
#pragma unroll
  for (int r = 0; r < 3; ++r) rv[r] = tf_of(rh[r], (TF *)nullptr);
  r2 += rv[0] * rv[0] + rv[1] * rv[1] + rv[2] * rv[2];
  const TF rbv[3] = {rv[0] * iwcc, rv[1] * iwcc, rv[2] * iwcc};
  combine<TF>(L, R, n, c1, c2, rbv, gh, full);
}

template <typename TF>
__device__ __forceinline__ void store_gh(float *slot_base, int lane, const TF gh[21]) {
  float *g = slot_base + lane;
#pragma unroll
  for (int q = 0; q < 21; ++q) g[q * 32] = gh[q];
}

// Bottom laminate i (leaves 2i, 2i+1) with strain e: leaf laws, its
// condensed record and plain stress sum; |r|^2, D and X accumulated.
template <typename TF, typename HP, int LAW>
__device__ __forceinline__ void laminate(WCtx<TF, HP> &c, int i, const HP e[6], Rec<TF> &rec, HP S[6],
                                         TF *gh) {
  const SolveParams &P = *c.P;
  NodeHP<HP> nd;
  load_node(P, i, nd);  // bottom laminate i is node i
  HP el[6], er[6];
  child_strains(nd, c.a_s + 3 * i, e, el, er);
  HP sl[6], sr[6], DL, DR, XL, XR;
  Rec<TF> rr;
  leaf_at<TF, HP, LAW>(c, 2 * i, el, sl, DL, XL, rec);
  leaf_at<TF, HP, LAW>(c, 2 * i + 1, er, sr, DR, XR, rr);
  HP *tag = nullptr;
  const HP wL = hp_from(__ldg(P.leafw + 2 * i), tag), wR = hp_from(__ldg(P.leafw + 2 * i + 1), tag);
  if (c.full) {
    c.Dsum = c.Dsum + (wL * DL + wR * DR);
    c.Xsum = c.Xsum + (wL * XL + wR * XR);
  }
  HP dsh[6];
#pragma unroll
  for (int q = 0; q < 6; ++q) {
    S[q] = wL * sl[q] + wR * sr[q];
    dsh[q] = sl[q] - sr[q];
  }
  HP rbh[3];
  btvec_hp(nd, dsh, rbh);  // B^T (sigma_L - sigma_R) = r_i / (w c1 c2)
  TF n[3], c1, c2, iwcc, wcc;
  load_node_tf(P, i, n, c1, c2, iwcc, wcc);
  TF rbv[3];
#pragma unroll
  for (int r = 0; r < 3; ++r) rbv[r] = tf_of(rbh[r], (TF *)nullptr);
  c.r2 += wcc * wcc * (rbv[0] * rbv[0] + rbv[1] * rbv[1] + rbv[2] * rbv[2]);
  combine<TF>(rec, rr, n, c1, c2, rbv, gh, c.full);
}

template <typename TF, typename HP>
__device__ __forceinline__ void rec_copy(Rec<TF> &d, const Rec<TF> &s) { d = s; }

// Condensed record (and plain stress sum) of lane l's subtree, the one under
// level-6 node l with strain e6.  Postorder over the lane's M bottom
// laminates: one copy of the laminate code and one of the code combining two
// subtrees (the instruction cache holds the loop); a record waiting for its
// sibling stays in the register slot of its level (at most two, K = 8), which
// the loop addresses by selects, never by an index.
template <int K, typename TF, typename HP, int LAW>
__device__ __forceinline__ void lane_condense(WCtx<TF, HP> &c, const HP e6[6], Rec<TF> &rec, HP S[6]) {
  constexpr int M = 1 << (K - 6);
  const SolveParams &P = *c.P;
  const int lane = c.lane;
  Rec<TF> pend0, pend1;  // waiting records of levels K and K - 1
  HP pS0[6], pS1[6];
#pragma unroll 1
  for (int q = 0; q < M; ++q) {
    // strain of bottom laminate lane M + q: down from level 6 along q's bits
    HP e[6];
#pragma unroll
    for (int c6 = 0; c6 < 6; ++c6) e[c6] = e6[c6];
#pragma unroll
    for (int lev = 6; lev < K; ++lev) {
      const int pos = (lane << (lev - 6)) + (q >> (K - lev));
      const int p = (1 << K) - (1 << lev) + pos;
      NodeHP<HP> nd;
      load_node(P, p, nd);
      const HP *a = c.a_s + 3 * p;
      const HP av[3] = {a[0], a[1], a[2]};
      HP J[6];
      bvec_hp(nd, av, J);
      const bool right = (q >> (K - lev - 1)) & 1;
#pragma unroll
      for (int c6 = 0; c6 < 6; ++c6) e[c6] = right ? e[c6] - nd.c1 * J[c6] : e[c6] + nd.c2 * J[c6];
    }
    TF gh[21];
    laminate<TF, HP, LAW>(c, lane * M + q, e, rec, S, gh);
    store_gh(c.ghw + DMN_IDX((M - 1) + q, 2 * M - 1) * 21 * 32, lane, gh);
    // merge with waiting left siblings while this record is a right child
    int lev = K, idx = q;
#pragma unroll 1
    while (idx & 1) {
      Rec<TF> L;
      HP SL[6];
      if (lev == K) {
        L = pend0;
#pragma unroll
        for (int c6 = 0; c6 < 6; ++c6) SL[c6] = pS0[c6];
      } else {
        L = pend1;
#pragma unroll
        for (int c6 = 0; c6 < 6; ++c6) SL[c6] = pS1[c6];
      }
      idx >>= 1;
      lev -= 1;
      const int p = (1 << K) - (1 << lev) + (lane << (lev - 6)) + idx;
      combine_node<TF, HP>(P, p, L, rec, SL, S, c.r2, c.full, gh);
      store_gh(c.ghw + DMN_IDX(((1 << (lev - 6)) - 1) + idx, 2 * M - 1) * 21 * 32, lane, gh);
      rec = L;
#pragma unroll
      for (int c6 = 0; c6 < 6; ++c6) S[c6] = SL[c6];
    }
    if (lev > 6) {  // a left child: wait for the sibling
      if (lev == K) {
        pend0 = rec;
#pragma unroll
        for (int c6 = 0; c6 < 6; ++c6) pS0[c6] = S[c6];
      } else {
        pend1 = rec;
#pragma unroll
        for (int c6 = 0; c6 < 6; ++c6) pS1[c6] = S[c6];
      }
    }
  }
}

// Back-substitution in the lane's subtree: node i of level LEV with the
// strain perturbation de from its ancestors.
template <int K, int LEV, typename TF, typename HP>
__device__ __forceinline__ void subtree_back(WCtx<TF, HP> &c, int i, const TF de[6]) {
  const SolveParams &P = *c.P;
  const int p = DMN_IDX((1 << K) - (1 << LEV) + i, (1 << K) - 1);
  const int slot = DMN_IDX(((1 << (LEV - 6)) - 1) + (i - (c.lane << (LEV - 6))), (1 << (K - 5)) - 1);
  const float *g = c.ghw + slot * 21 * 32 + c.lane;
  TF gh[21];
#pragma unroll
  for (int q = 0; q < 21; ++q) gh[q] = g[q * 32];
  TF da[3];
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    TF s = gh[18 + r];
#pragma unroll
    for (int q = 0; q < 6; ++q) s += gh[6 * r + q] * de[q];
    da[r] = -s;
  }
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    c.da_s[3 * p + r] = da[r];
    c.a_s[3 * p + r] = hp_add_tf(c.a_s[3 * p + r], da[r]);
  }
  if constexpr (LEV < K) {
    TF n[3], c1, c2, iwcc, wcc;
    load_node_tf(P, p, n, c1, c2, iwcc, wcc);
    TF J[6], dl[6], dr[6];
    bvec(n, da, J);
#pragma unroll
    for (int q = 0; q < 6; ++q) {
      dl[q] = de[q] + c2 * J[q];
      dr[q] = de[q] - c1 * J[q];
    }
    subtree_back<K, LEV + 1, TF, HP>(c, 2 * i, dl);
    subtree_back<K, LEV + 1, TF, HP>(c, 2 * i + 1, dr);
  }
}

// traces of the leaf strains at t^n under node i of level LEV (trace tr):
// tr(B a) = a . n
template <int K, int LEV, typename HP>
__device__ __forceinline__ void subtree_traces(const SolveParams &P, const HP *a_s, HP *trn_s, int i, HP tr) {
  const int p = (1 << K) - (1 << LEV) + i;
  NodeHP<HP> nd;
  load_node(P, p, nd);
  const HP *a = a_s + 3 * p;
  const HP t = a[0] * nd.n[0] + a[1] * nd.n[1] + a[2] * nd.n[2];
  const HP tl = tr + nd.c2 * t, trr = tr - nd.c1 * t;
  if constexpr (LEV == K) {
    trn_s[2 * i] = tl;
    trn_s[2 * i + 1] = trr;
  } else {
    subtree_traces<K, LEV + 1, HP>(P, a_s, trn_s, 2 * i, tl);
    subtree_traces<K, LEV + 1, HP>(P, a_s, trn_s, 2 * i + 1, trr);
  }
}

// strain (or trace) of lane l's level-6 node from the root value: the five
// upper ancestors' terms, root first (+c2 B a on the way to child 1, -c1 B a
// to child 2)
template <int K, typename HP>
__device__ __forceinline__ void level6_strain(const SolveParams &P, const HP *a_s, int l, const HP root[6],
                                              HP e[6]) {
#pragma unroll
  for (int q = 0; q < 6; ++q) e[q] = root[q];
#pragma unroll
  for (int k = 1; k <= 5; ++k) {
    const int i = l >> (6 - k), p = (1 << K) - (1 << k) + i;
    const bool right = (l >> (5 - k)) & 1;
    NodeHP<HP> nd;
    load_node(P, p, nd);
    const HP av[3] = {a_s[3 * p], a_s[3 * p + 1], a_s[3 * p + 2]};
    HP J[6];
    bvec_hp(nd, av, J);
#pragma unroll
    for (int q = 0; q < 6; ++q) e[q] = right ? e[q] - nd.c1 * J[q] : e[q] + nd.c2 * J[q];
  }
}
template <int K, typename HP>
__device__ __forceinline__ HP level6_trace(const SolveParams &P, const HP *a_s, int l, HP tr) {
#pragma unroll
  for (int k = 1; k <= 5; ++k) {
    const int i = l >> (6 - k), p = (1 << K) - (1 << k) + i;
    const bool right = (l >> (5 - k)) & 1;
    NodeHP<HP> nd;
    load_node(P, p, nd);
    const HP t = a_s[3 * p] * nd.n[0] + a_s[3 * p + 1] * nd.n[1] + a_s[3 * p + 2] * nd.n[2];
    tr = right ? tr - nd.c1 * t : tr + nd.c2 * t;
  }
  return tr;
}

template <typename TF>
__device__ __forceinline__ void rec_shfl(Rec<TF> &dst, const Rec<TF> &src, int off) {
  rec_shfl_down(dst, src, off, kFull, 32);
}

}  // namespace warp_detail

// Shared buffers of the batched upper levels, after the W per-warp regions:
// level-5 records and plain stress sums of every point (slot pw 16 + j; level
// 3 reuses them), level 4 (slot pw 8 + j; level 2 reuses them), the roots,
// per-node |r|^2 of levels 4..1 (pw 16 + 16 - 2^k + j), per-warp |r|^2 of
// the lane levels and level 5, per-point flags (1: active, 2: full pass).
namespace warp_detail {
constexpr int RSW = 41;  // record stride in floats (40 values, odd)
__host__ __device__ constexpr int up_rec5(int) { return 0; }                             // TF[W 16 RSW]
__host__ __device__ constexpr int up_s5(int W) { return 4 * W * 16 * RSW + 4 * (W & 1); }  // HP[W 16 6]
__host__ __device__ constexpr int up_rec4(int W) { return up_s5(W) + 8 * W * 16 * 6; }    // TF[W 8 RSW]
__host__ __device__ constexpr int up_s4(int W) { return up_rec4(W) + 4 * W * 8 * RSW + 4 * (W & 1); }  // HP
__host__ __device__ constexpr int up_root(int W) { return up_s4(W) + 8 * W * 8 * 6; }     // TF[W RSW]
__host__ __device__ constexpr int up_sroot(int W) { return (up_root(W) + 4 * W * RSW + 7) & ~7; }  // HP[W 6]
__host__ __device__ constexpr int up_r2(int W) { return up_sroot(W) + 8 * W * 6; }        // TF[W 16]
__host__ __device__ constexpr int up_r2w(int W) { return up_r2(W) + 4 * W * 16; }         // TF[W]
__host__ __device__ constexpr int up_flag(int W) { return up_r2w(W) + 4 * W; }            // int[W]
__host__ __device__ constexpr int up_bytes(int W) { return (up_flag(W) + 4 * W + 15) & ~15; }

template <typename TF>
__device__ __forceinline__ void rec_to_smem(TF *d, const Rec<TF> &r) {
#pragma unroll
  for (int q = 0; q < 21; ++q) d[q] = r.C[q];
#pragma unroll
  for (int c = 0; c < 6; ++c) {
    d[21 + c] = r.ds[c];
    d[27 + c] = r.tau[c];
    d[33 + c] = r.dd[c];
  }
  d[39] = r.gg;
}
template <typename TF>
__device__ __forceinline__ void rec_from_smem(Rec<TF> &r, const TF *d) {
#pragma unroll
  for (int q = 0; q < 21; ++q) r.C[q] = d[q];
#pragma unroll
  for (int c = 0; c < 6; ++c) {
    r.ds[c] = d[21 + c];
    r.tau[c] = d[27 + c];
    r.dd[c] = d[33 + c];
  }
  r.gg = d[39];
}
}  // namespace warp_detail

// K: depth (6..8); W: warps (points) per CTA (4: levels 4..1 of all points fit
// one warp); MINB: CTAs per SM the register budget is sized for; LAW as in the
// compact form (1: thermoelastic and J2 leaves).  Mixed precision only
// (TF = float, HP = float-float).
//
// The W warps of a CTA run their passes in lockstep, one pass per slot:
//   [A] a warp without a point takes one from the queue and loads it;
//   [C] every warp condenses its point's level-6 subtrees (a lane each) and
//       level 5 (lane pairs, shuffles);
//   [E] warp 0 condenses levels 4..1 of all W points, one node per lane;
//   [G] every warp takes Algorithm 1's decision for its point and makes the
//       Newton step, the line-search step, or writes the outputs.
// Barriers between [C], [E] and [G] keep the warps of a CTA in the same code,
// which the instruction cache needs; the batched phase [E] condenses the
// upper levels of W points for the price of one.
template <int K, int W, int MINB, int LAW>
__global__ void __launch_bounds__(32 * W, MINB) dmn_solve_warp(const SolveParams P) {
  using namespace warp_detail;
  using TF = float;
  using HP = dfl;
  constexpr int N = (1 << K) - 1;
  static_assert(W * 8 <= 32, "levels 4..1 of all points on one warp");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  HP *tag = nullptr;
  MatPt<TF, HP> *mp_static = reinterpret_cast<MatPt<TF, HP> *>(smem_raw);
  const int wbytes = wlay_bytes(K, P.n_mats, int(sizeof(MatPt<TF, HP>)));
  unsigned char *wbase0 = smem_raw + ((P.n_mats * int(sizeof(MatPt<TF, HP>)) + 15) & ~15);
  unsigned char *wbase = wbase0 + warp * wbytes;
  unsigned char *ubase = wbase0 + W * wbytes;
  HP *a_s = reinterpret_cast<HP *>(wbase + wlay_a(K));
  HP *e6_s = reinterpret_cast<HP *>(wbase + wlay_e6(K));
  HP *trn_s = reinterpret_cast<HP *>(wbase + wlay_trn(K));
  HP *eb = reinterpret_cast<HP *>(wbase + wlay_eb(K));  // eps_bar^{n+1} (HP), deps (HP)
  double *ebd = reinterpret_cast<double *>(wbase + wlay_eb(K) + 8 * 12);  // eps_bar^{n+1} (FP64)
  HP *ohp = reinterpret_cast<HP *>(wbase + wlay_out(K));                  // D_bar, X_bar
  TF *da_s = reinterpret_cast<TF *>(wbase + wlay_da(K));
  TF *ghu = reinterpret_cast<TF *>(wbase + wlay_ghu(K));
  MatPt<TF, HP> *mp = reinterpret_cast<MatPt<TF, HP> *>(wbase + wlay_mat(K));
  TF *rec5 = reinterpret_cast<TF *>(ubase + up_rec5(W));
  HP *s5 = reinterpret_cast<HP *>(ubase + up_s5(W));
  TF *rec4 = reinterpret_cast<TF *>(ubase + up_rec4(W));
  HP *s4 = reinterpret_cast<HP *>(ubase + up_s4(W));
  TF *rootr = reinterpret_cast<TF *>(ubase + up_root(W));
  HP *sroot = reinterpret_cast<HP *>(ubase + up_sroot(W));
  TF *r2up = reinterpret_cast<TF *>(ubase + up_r2(W));
  TF *r2w = reinterpret_cast<TF *>(ubase + up_r2w(W));
  int *pflag = reinterpret_cast<int *>(ubase + up_flag(W));
  float *ghw = P.gh + size_t(blockIdx.x * W + warp) * wscratch_floats(K);

  for (int i = threadIdx.x; i < P.n_mats; i += 32 * W)
    mat_static<TF, HP>(mp_static[i], *reinterpret_cast<const MatDev *>(P.mat + kMatWords * i), P.dt);
  __syncthreads();
  const HP idt = hp_from(1.0 / P.dt, tag);
  const TF idt_f = TF(1.0 / P.dt);
  const TF tol = TF(P.tol), res_floor = TF(P.res_floor), gamma = TF(P.gamma);
  constexpr int pu0 = (1 << K) - 32;  // first node of level 5

  WCtx<TF, HP> c;
  c.P = &P;
  c.a_s = a_s;
  c.da_s = da_s;
  c.trn_s = trn_s;
  c.mp = mp;
  c.ghw = ghw;
  c.lane = lane;
  // the warp's point and its Algorithm 1 state (identical on every lane)
  bool active = false, exhausted = false, first = true;
  int64_t pt = 0;
  double theta = 0.0;
  int it = 0, bt = 0, status = 0, attempt = 0, it_total = 0;
  TF gi = TF(1), res_old = TF(0);
  Rec<TF> rec;
  HP S[6];

  for (;;) {
    // ---- [A] a warp without a point takes the next one and loads it
    if (!active && !exhausted) {
      unsigned long long q = 0;
      if (lane == 0) {
        q = atomicAdd(P.queue, 1ull);
        while (P.skip && q < (unsigned long long)P.n_points && P.skip[q] != 0) q = atomicAdd(P.queue, 1ull);
      }
      q = __shfl_sync(kFull, q, 0);
      if (q >= (unsigned long long)P.n_points) {
        exhausted = true;
      } else {
        active = true;
        pt = int64_t(q);
        DMN_BOUNDS_CLEAR();
        const double *sin = P.sin + pt * P.SW;
        c.sin = sin;
        c.sout = P.sout + pt * P.SW;
        theta = P.theta[pt];
        if (lane < 6) {
          const double e0 = ld_stream(sin + lane), d = ld_stream(P.deps + pt * 6 + lane);
          ebd[lane] = e0 + d;  // eps_bar^{n+1} = eps_bar^n + deps exactly in FP64
          eb[lane] = hp_load(e0 + d, tag);
          eb[6 + lane] = hp_load(d, tag);
        }
        for (int i = lane; i < 3 * N; i += 32) a_s[i] = hp_load(ld_stream(sin + 8 + i), tag);
        if (lane < P.n_mats) {
          mp[lane] = mp_static[lane];
          mat_point<TF, HP, LAW>(mp[lane], hp_load(theta, tag), idt, idt_f);
        }
        __syncwarp();
        {
          // traces of the leaf strains at t^n (the coupling term needs tr eps^n)
          const HP tr0 = hp_load(ld_stream(sin), tag) + hp_load(ld_stream(sin + 1), tag) +
                         hp_load(ld_stream(sin + 2), tag);
          subtree_traces<K, 6, HP>(P, a_s, trn_s, lane, level6_trace<K, HP>(P, a_s, lane, tr0));
        }
        __syncwarp();
        if (P.da0) {  // warm start a^n + da0
          const float *d0 = P.da0 + pt * (3 * N);
          for (int i = lane; i < 3 * N; i += 32) a_s[i] = hp_add_tf(a_s[i], ld_stream(d0 + i));
          __syncwarp();
        }
        HP e[6];
        level6_strain<K, HP>(P, a_s, lane, eb, e);
#pragma unroll
        for (int q2 = 0; q2 < 6; ++q2) e6_s[6 * lane + q2] = e[q2];
        first = true;
        it = bt = status = attempt = it_total = 0;
        gi = TF(1);
        res_old = TF(0);
      }
    }
    if (lane == 0) pflag[warp] = (active ? 1 : 0) | (first ? 0 : 2);
    if (!__syncthreads_or(active)) break;

    // ---- [C] the lanes' subtrees and level 5
    if (active) {
      // Algorithm 1 takes at least one Newton step, so the first pass of an
      // iteration never gives the outputs: it skips their terms
      c.full = !first;
      c.r2 = TF(0);
      c.Dsum = hp_zero(tag);
      c.Xsum = hp_zero(tag);
      {
        HP e[6];
#pragma unroll
        for (int q2 = 0; q2 < 6; ++q2) e[q2] = e6_s[6 * lane + q2];
        lane_condense<K, TF, HP, LAW>(c, e, rec, S);
      }
      Rec<TF> other;
      rec_shfl(other, rec, 1);
      HP So[6];
#pragma unroll
      for (int q2 = 0; q2 < 6; ++q2) So[q2] = hp_shfl_down(kFull, S[q2], 1, 32);
      if ((lane & 1) == 0) {
        const int j = lane >> 1, p = pu0 + j;
        combine_node<TF, HP>(P, p, rec, other, S, So, c.r2, c.full, ghu + 21 * DMN_IDX(p - pu0, kUpNodes));
        rec_to_smem(rec5 + RSW * (warp * 16 + j), rec);
#pragma unroll
        for (int q2 = 0; q2 < 6; ++q2) s5[6 * (warp * 16 + j) + q2] = S[q2];
      }
      TF r2 = c.r2;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) r2 += __shfl_xor_sync(kFull, r2, o);
      if (lane == 0) r2w[warp] = r2;
    }
    __syncthreads();

    // ---- [E] levels 4..1 of every point on warp 0: level k node j of point
    //      pw on lane pw 2^(k-1) + j; children from the level below
    if (warp == 0) {
#pragma unroll 1
      for (int k = 4; k >= 1; --k) {
        const int cnt = 1 << (k - 1);
        const int pw = lane >> (k - 1), j = lane & (cnt - 1);
        if (pw < W && (pflag[pw] & 1)) {
          // level k + 1 lives in the level-5 slots (k + 1 odd) or the level-4 slots
          const bool from5 = ((k + 1) & 1) != 0;
          const TF *rb = from5 ? rec5 + RSW * (pw * 16) : rec4 + RSW * (pw * 8);
          const HP *sb = from5 ? s5 + 6 * (pw * 16) : s4 + 6 * (pw * 8);
          const int jl = DMN_IDX(2 * j, from5 ? 15 : 7);  // both children inside the buffer
          Rec<TF> L, R;
          rec_from_smem(L, rb + RSW * jl);
          rec_from_smem(R, rb + RSW * (jl + 1));
          HP SL[6], SR[6];
#pragma unroll
          for (int q2 = 0; q2 < 6; ++q2) {
            SL[q2] = sb[6 * jl + q2];
            SR[q2] = sb[6 * (jl + 1) + q2];
          }
          const int p = (1 << K) - (1 << k) + j;
          TF *ghu_pw = reinterpret_cast<TF *>(wbase0 + pw * wbytes + wlay_ghu(K));
          TF r2n = TF(0);
          combine_node<TF, HP>(P, p, L, R, SL, SR, r2n, (pflag[pw] & 2) != 0,
                               ghu_pw + 21 * DMN_IDX(p - pu0, kUpNodes));
          r2up[pw * 16 + DMN_IDX(16 - (1 << k) + j, 15)] = r2n;
          TF *rd;
          HP *sd;
          if (k == 1) {
            rd = rootr + RSW * pw;
            sd = sroot + 6 * pw;
          } else if (k & 1) {  // levels 3: the level-5 slots are free again
            rd = rec5 + RSW * (pw * 16 + DMN_IDX(j, 16));
            sd = s5 + 6 * (pw * 16 + DMN_IDX(j, 16));
          } else {
            rd = rec4 + RSW * (pw * 8 + DMN_IDX(j, 8));
            sd = s4 + 6 * (pw * 8 + DMN_IDX(j, 8));
          }
          rec_to_smem(rd, L);
#pragma unroll
          for (int q2 = 0; q2 < 6; ++q2) sd[q2] = SL[q2];
        }
        __syncwarp();
      }
    }
    __syncthreads();

    // ---- [G] decision (Algorithm 1), then the Newton step, the line-search
    //      step, or the outputs
    if (active) {
      TF r2 = r2w[warp];
#pragma unroll
      for (int i = 0; i < 15; ++i) r2 += r2up[warp * 16 + i];
      TF sn = TF(0);
#pragma unroll
      for (int q2 = 0; q2 < 6; ++q2) sn += sroot[6 * warp + q2].hi * sroot[6 * warp + q2].hi;
      TF den = sqrt(sn);
      if (den < res_floor) den = res_floor;
      const TF res = sqrt(r2) / (TF(N) * den);
      const bool accept = first || (res < res_old) || (bt >= P.maxbt);
      int action;
      if (accept) {
        if (!isfinite(res)) {
          status = 2;
          action = ACT_DONE;
        } else if (!first && res < tol) {
          status = 0;
          action = ACT_DONE;
        } else if (it >= P.maxit) {
          status = 1;
          action = ACT_DONE;
        } else {
          res_old = res;
          it += 1;
          bt = 0;
          gi = TF(1);
          action = ACT_STEP;
        }
        first = false;
      } else {
        action = ACT_BACK;
      }
      const double *sin = c.sin;
      double *sout = c.sout;
      if (action == ACT_DONE && P.da0 && attempt == 0 && status != 0) {
        // the warm-started iteration failed: Algorithm 1 again from a^n
        attempt = 1;
        it_total = it;
        for (int i = lane; i < 3 * N; i += 32) a_s[i] = hp_load(ld_stream(sin + 8 + i), tag);
        __syncwarp();
        HP e[6];
        level6_strain<K, HP>(P, a_s, lane, eb, e);
#pragma unroll
        for (int q2 = 0; q2 < 6; ++q2) e6_s[6 * lane + q2] = e[q2];
        first = true;
        it = bt = status = 0;
        gi = TF(1);
        res_old = TF(0);
      } else if (action == ACT_STEP) {
        // back-substitution: levels 1..5 by shuffles (the node's strain
        // perturbation de in TF for the Newton chain and the float-float sum
        // he of its ancestors' B da terms for the level-6 strain), then the
        // lane's own subtree
        TF de[6] = {TF(0), TF(0), TF(0), TF(0), TF(0), TF(0)};
        HP he[6];
#pragma unroll
        for (int q2 = 0; q2 < 6; ++q2) he[q2] = hp_zero(tag);
#pragma unroll 1
        for (int k = 1; k <= 5; ++k) {
          const int stride = 1 << (6 - k), half = stride >> 1;
          TF dr[6];
          HP hr[6];
          if ((lane & (stride - 1)) == 0) {
            const int j = lane >> (6 - k), p = (1 << K) - (1 << k) + j;
            const TF *g = ghu + 21 * DMN_IDX(p - pu0, kUpNodes);
            TF da[3];
#pragma unroll
            for (int r = 0; r < 3; ++r) {
              TF s2 = g[18 + r];
#pragma unroll
              for (int q2 = 0; q2 < 6; ++q2) s2 += g[6 * r + q2] * de[q2];
              da[r] = -s2;
            }
#pragma unroll
            for (int r = 0; r < 3; ++r) {
              da_s[3 * p + r] = da[r];
              a_s[3 * p + r] = hp_add_tf(a_s[3 * p + r], da[r]);
            }
            NodeHP<HP> nd;
            TF n[3], c1, c2, iwcc, wcc;
            node_all(P, p, nd, n, c1, c2, iwcc, wcc);
            TF J[6];
            bvec(n, da, J);
            const HP dah[3] = {hp_add_tf(hp_zero(tag), da[0]), hp_add_tf(hp_zero(tag), da[1]),
                               hp_add_tf(hp_zero(tag), da[2])};
            HP Jh[6];
            bvec_hp(nd, dah, Jh);
#pragma unroll
            for (int q2 = 0; q2 < 6; ++q2) {
              dr[q2] = de[q2] - c1 * J[q2];
              de[q2] = de[q2] + c2 * J[q2];
              hr[q2] = he[q2] - nd.c1 * Jh[q2];
              he[q2] = he[q2] + nd.c2 * Jh[q2];
            }
          }
          const bool recv = (lane & (stride - 1)) == half;
#pragma unroll
          for (int q2 = 0; q2 < 6; ++q2) {
            const TF v = __shfl_up_sync(kFull, dr[q2], half);
            const float vh = __shfl_up_sync(kFull, hr[q2].hi, half);
            const float vl = __shfl_up_sync(kFull, hr[q2].lo, half);
            if (recv) {
              de[q2] = v;
              he[q2] = {vh, vl};
            }
          }
        }
#pragma unroll
        for (int q2 = 0; q2 < 6; ++q2) e6_s[6 * lane + q2] = e6_s[6 * lane + q2] + he[q2];
        subtree_back<K, 6, TF, HP>(c, lane, de);
      } else if (action == ACT_BACK) {
        // backtracking (rare): a -= f da, strains again from a
        const TF f = gi * (TF(1) - gamma);
        for (int i = lane; i < 3 * N; i += 32) a_s[i] = hp_add_tf(a_s[i], -f * da_s[i]);
        __syncwarp();
        HP e[6];
        level6_strain<K, HP>(P, a_s, lane, eb, e);
#pragma unroll
        for (int q2 = 0; q2 < 6; ++q2) e6_s[6 * lane + q2] = e[q2];
        gi *= gamma;
        bt += 1;
      } else {
        // ---- outputs and state (the last pass is at the final a)
        HP Db = c.Dsum, Xb = c.Xsum;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          Db = Db + hp_shfl_down(kFull, Db, o, 32);
          Xb = Xb + hp_shfl_down(kFull, Xb, o, 32);
        }
        if (lane == 0) {
          ohp[0] = Db;
          ohp[1] = Xb;
        }
        __syncwarp();
        const TF *orr = rootr + RSW * warp;
        const HP *osg = sroot + 6 * warp;
        int bad = 0;
        for (int cc = lane; cc < kOutWords; cc += 32) {
          double v;
          if (cc < 6) v = hp_to(osg[cc]);
          else if (cc < 42) v = double(sget(orr, (cc - 6) / 6, (cc - 6) % 6));
          else if (cc < 48) v = double(orr[27 + cc - 42]);   // tau
          else if (cc == 48) v = hp_to(ohp[0]);
          else if (cc < 55) v = double(orr[33 + cc - 49]);   // dd
          else if (cc == 55) v = double(orr[39]);            // gg
          else v = hp_to(ohp[1]);
          if (!isfinite(v)) bad = 1;
          __stcs(P.out + pt * kOutWords + cc, v);
        }
        bad = __any_sync(kFull, bad);
        const int bbad = DMN_BOUNDS_GET();
        if (lane == 0) {
          P.status[pt] = (bad ? 2 : status) | (attempt ? 4 : 0) | (bbad ? kPtBounds : 0);
          P.iters[pt] = it + it_total;
        }
        if (lane < 8) sout[lane] = lane < 6 ? ebd[lane] : (lane == 6 ? theta : 0.0);
        for (int i = lane; i < 3 * N; i += 32) __stcs(sout + 8 + i, hp_to(a_s[i]));
        // the lane's own leaves: parked float-float z of the last pass -> FP64
#pragma unroll 1
        for (int j = lane << (K - 5); j < (lane + 1) << (K - 5); ++j) {
          const int zo = __ldg(P.zoff + j);
          if (zo < 0) continue;
          const int nz = (LAW >= 2 && mp[__ldg(P.phase + j)].kind == 2) ? 13 : 7;
          const HP *zp = reinterpret_cast<const HP *>(sout + zo);
          for (int q2 = 0; q2 < nz; ++q2) {
            const HP v = ld_once(zp + q2);
            sout[zo + q2] = hp_to(v);
          }
        }
        for (int i = P.zend + lane; i < P.SW; i += 32) sout[i] = 0.0;  // padding word
        active = false;
      }
      __syncwarp();
    }
  }
}

}  // namespace dmn
