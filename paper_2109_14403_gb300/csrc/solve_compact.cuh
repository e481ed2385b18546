// solve_compact.cuh -- second form of the Algorithm 1 solve (arXiv
// 2109.14403, Sec. 3.3): one CTA per Gauss point, G = 2^(K-1) threads, with
//  * incremental strains: the strains of the bottom laminates live in shared
//    memory and are updated after each Newton step by adding, in the high
//    precision HP (float-float in the mixed path), the strain increments the
//    exact FP32 jump increments da cause (eq. DMN kinematics);
//  * strain sums instead of level sweeps: a bottom laminate's strain (or
//    increment) is the root value plus one term per ancestor; all terms are
//    formed at once, one node per thread, and summed per laminate after a
//    single barrier;
//  * compact levels: the laminates just above the bottom pair neighbouring
//    lanes by shuffle; every higher level condenses node j on eight lanes,
//    one Mandel row each (combine_rows), with the children's condensed
//    records and stress sums in shared memory, so a level of at most four
//    nodes occupies one warp (the CTA's leader warp, with warp barriers
//    only) while the other warps go ahead;
//  * the back-substitution of the Newton increment, a chain through the
//    levels, in the condensation precision TF on the same compact mapping;
//  * the point's state block (jumps, internal variables) brought into shared
//    memory by the bulk-copy engine and converted in place by short loops.
// The leader warp is picked from the CTA's warp slot so that the CTAs resident
// on one SM run their single-warp phases on different SM sub-partitions.
// The condensation, the residual and the leaf laws are those of
// dmn_kernels.cuh.  The internal variables of the current pass are parked in
// the caller's output state (same 8-byte slots) and converted at the end.
#pragma once
#include "dmn_internal.h"
#include "solve_common.cuh"
#include "pa66.cuh"

namespace dmn {

namespace compact_detail {
constexpr int RS = 41;  // record stride in shared memory (40 values, odd)

template <typename TF>
__device__ __forceinline__ void rec_put(TF *s, const Rec<TF> &r) {
#pragma unroll
  for (int q = 0; q < 21; ++q) s[q] = r.C[q];
#pragma unroll
  for (int c = 0; c < 6; ++c) {
    s[21 + c] = r.ds[c];
    s[27 + c] = r.tau[c];
    s[33 + c] = r.dd[c];
  }
  s[39] = r.gg;
}
template <typename TF>
__device__ __forceinline__ void rec_get(Rec<TF> &r, const TF *s) {
#pragma unroll
  for (int q = 0; q < 21; ++q) r.C[q] = s[q];
#pragma unroll
  for (int c = 0; c < 6; ++c) {
    r.ds[c] = s[21 + c];
    r.tau[c] = s[27 + c];
    r.dd[c] = s[33 + c];
  }
  r.gg = s[39];
}

template <typename T>
__device__ __forceinline__ T pick3(const T v[3], int i) {
  return i == 0 ? v[0] : (i == 1 ? v[1] : v[2]);
}

// The condensation of node p (combine() of dmn_kernels.cuh, the same
// formulas) by an aligned group of eight lanes: lane r < 6 owns Mandel row r
// of the tangents and component r of the vectors; lanes 6 and 7 repeat row 5
// and store nothing.  B^T couples traction component e with rows e, ra(e),
// rb(e) (t_e = s_e n_e + (s_ra n_ia + s_rb n_ib) / sqrt2), so lane e < 3
// gathers those two rows by shuffles to form row e of K = B^T M B and the
// components e of the right-hand sides; everything 3-wide is then broadcast.
// rcL, rcR: the children's records; sL, sR: their stress sums (HP).  With
// st, writes the node's record (root: the output layout of orec, C, tau at
// 21, dd at 27, g at 33) into dst, its stress sum into sdst, G_p and h_p
// into gh, and adds the lane's part of |r_p|^2 to r2.
template <typename TF, typename HP>
__device__ __forceinline__ void combine_rows(const SolveParams &P, int p, int r, bool st, unsigned mask,
                                             const TF *rcL, const TF *rcR, const HP *sL, const HP *sR,
                                             TF *dst, HP *sdst, TF *gh, TF &r2, bool full, bool root) {
  const int rw = r < 6 ? r : 5;
  const int ra = rw == 2 ? 4 : 5, rb = rw == 0 ? 4 : 3;  // rows coupled with component e = rw < 3
  const int ia = rw == 0 ? 1 : 0, ib = rw == 2 ? 1 : 2;
  const bool own = st && r < 6;
  auto sh = [&](TF v, int src) { return __shfl_sync(mask, v, src, 8); };
  TF n[3], c1, c2, iwcc, wcc;
  load_node_tf(P, p, n, c1, c2, iwcc, wcc);
  const TF rs = TF(kRsq2);
  const TF ne = pick3(n, rw), na = pick3(n, ia), nb = pick3(n, ib);
  const TF cc = c1 * c2;
  // traction component e = rw of a Mandel vector whose component rw is v
  auto bt_e = [&](TF v) { return v * ne + rs * (sh(v, ra) * na + sh(v, rb) * nb); };

  // row rw of M = c2 C_L + c1 C_R and of dC = C_L - C_R
  const int rbase = rw * (11 - rw) / 2;  // packed index of (rw, rw) minus rw
  TF M[6], dC[6];
#pragma unroll
  for (int c = 0; c < 6; ++c) {
    const int q = c >= rw ? rbase + c : c * (11 - c) / 2 + rw;
    const TF cl = rcL[q], cr = rcR[q];
    M[c] = c2 * cl + c1 * cr;
    dC[c] = cl - cr;
  }
  // row rw of M B and of U = dC B; row e of K on lane e < 3, then all of K
  TF MB[3], U[3];
  btvec(n, M, MB);
  btvec(n, dC, U);
  TF Kr[3];
#pragma unroll
  for (int f = 0; f < 3; ++f) Kr[f] = bt_e(MB[f]);
  const TF k00 = sh(Kr[0], 0), k11 = sh(Kr[1], 1), k22 = sh(Kr[2], 2);
  const TF k01 = TF(0.5) * (sh(Kr[1], 0) + sh(Kr[0], 1));
  const TF k02 = TF(0.5) * (sh(Kr[2], 0) + sh(Kr[0], 2));
  const TF k12 = TF(0.5) * (sh(Kr[2], 1) + sh(Kr[1], 2));
  const TF a00 = k11 * k22 - k12 * k12, a01 = k02 * k12 - k01 * k22, a02 = k01 * k12 - k02 * k11;
  const TF a11 = k00 * k22 - k02 * k02, a12 = k01 * k02 - k00 * k12, a22 = k00 * k11 - k01 * k01;
  const TF idet = TF(1) / (k00 * a00 + k01 * a01 + k02 * a02);
  const TF Ki[3][3] = {{a00 * idet, a01 * idet, a02 * idet},
                       {a01 * idet, a11 * idet, a12 * idet},
                       {a02 * idet, a12 * idet, a22 * idet}};
  // column rw of G = K^{-1} U^T
  TF V[3];
#pragma unroll
  for (int e = 0; e < 3; ++e) V[e] = Ki[e][0] * U[0] + Ki[e][1] * U[1] + Ki[e][2] * U[2];
  if (own) {
#pragma unroll
    for (int e = 0; e < 3; ++e) gh[6 * e + r] = V[e];
  }
  // residual r_p = w c1 c2 B^T (c2 S_L - c1 S_R) in HP; component e on lane e
  HP S;
  TF rbv_e;
  {
    NodeHP<HP> nd;
    load_node(P, p, nd);
    const HP SL = sL[rw], SR = sR[rw];
    S = SL + SR;
    const HP dh = nd.c2 * SL - nd.c1 * SR;
    const HP dha = hp_shfl(mask, dh, ra, 8), dhb = hp_shfl(mask, dh, rb, 8);
    const HP rh = dh * pick3(nd.n, rw) + dha * pick3(nd.ns, ia) + dhb * pick3(nd.ns, ib);
    const TF rv = tf_of(rh, (TF *)nullptr);
    if (st && r < 3) r2 += rv * rv;
    rbv_e = rv * iwcc;
  }
  // condensed stress: B^T ds_hat = rb + B^T (ds_L - ds_R)
  const TF dsL = rcL[21 + rw], dsR = rcR[21 + rw];
  const TF b3e = rbv_e + bt_e(dsL - dsR);
  const TF b3[3] = {sh(b3e, 0), sh(b3e, 1), sh(b3e, 2)};
  TF hs[3];
#pragma unroll
  for (int e = 0; e < 3; ++e) hs[e] = Ki[e][0] * b3[0] + Ki[e][1] * b3[1] + Ki[e][2] * b3[2];
  if (st && r == 0) {
#pragma unroll
    for (int e = 0; e < 3; ++e) gh[18 + e] = hs[e];
  }
  const TF ds = c1 * dsL + c2 * dsR - cc * (U[0] * hs[0] + U[1] * hs[1] + U[2] * hs[2]);
  TF tau = TF(0), dd = TF(0), gg = TF(0);
  if (full) {
    const TF tL = rcL[27 + rw], tR = rcR[27 + rw], dL = rcL[33 + rw], dR = rcR[33 + rw];
    const TF te = bt_e(tL - tR), de = bt_e(dL - dR);
    const TF t3[3] = {sh(te, 0), sh(te, 1), sh(te, 2)};
    const TF bd[3] = {sh(de, 0), sh(de, 1), sh(de, 2)};
    TF ht[3], hd[3];
#pragma unroll
    for (int e = 0; e < 3; ++e) {
      ht[e] = Ki[e][0] * t3[0] + Ki[e][1] * t3[1] + Ki[e][2] * t3[2];
      hd[e] = Ki[e][0] * bd[0] + Ki[e][1] * bd[1] + Ki[e][2] * bd[2];
    }
    // g_hat = c1 g_L + c2 g_R - c1 c2 (B^T d_diff) . h_tau
    gg = c1 * rcL[39] + c2 * rcR[39] - cc * (bd[0] * ht[0] + bd[1] * ht[1] + bd[2] * ht[2]);
    tau = c1 * tL + c2 * tR - cc * (U[0] * ht[0] + U[1] * ht[1] + U[2] * ht[2]);
    dd = c1 * dL + c2 * dR - cc * (U[0] * hd[0] + U[1] * hd[1] + U[2] * hd[2]);
  }
  // row rw of C_hat = c1 C_L + c2 C_R - c1 c2 U G, c1 C_L + c2 C_R = M + (c1 - c2) dC
  const TF cm = c1 - c2;
#pragma unroll
  for (int c = 0; c < 6; ++c) {
    const TF g0 = sh(V[0], c), g1 = sh(V[1], c), g2 = sh(V[2], c);
    const TF v = M[c] + cm * dC[c] - cc * (U[0] * g0 + U[1] * g1 + U[2] * g2);
    if (own && c >= rw) dst[rbase + c] = v;
  }
  if (own) {
    sdst[r] = S;
    if (root) {
      if (full) {
        dst[21 + r] = tau;
        dst[27 + r] = dd;
        if (r == 0) dst[33] = gg;
      }
    } else {
      dst[21 + r] = ds;
      if (full) {
        dst[27 + r] = tau;
        dst[33 + r] = dd;
        if (r == 0) dst[39] = gg;
      }
    }
  }
}

// The state block of a point is moved into shared memory by the bulk-copy
// engine (cp.async.bulk, completion counted on an mbarrier): the jumps a into
// a_s and, for the kinds that keep their internal variables as stored, z into
// zn_s; each thread then converts its words in place.  A block has an even
// number of words and starts on a 16-byte boundary, so a (word 8) starts
// aligned and goes with the word after it (3N is odd), and z (word 8 + 3N,
// odd) goes from the word before it into the slot before zn_s, rounded up to
// an even count.  The extra words stay inside the block and land in slots
// written before they are read (eK[0], eK[6G - 1], eb[0]).
constexpr int kWaitLimit = 1 << 22;  // mbarrier polls before a point gives up
__device__ __forceinline__ unsigned smem_u32(const void *p) {
  return unsigned(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void bulk_g2s(unsigned dst, const void *src, unsigned bytes, unsigned mb) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
               ::"r"(dst), "l"(src), "r"(bytes), "r"(mb)
               : "memory");
}
// poll the mbarrier's phase with the given parity, at most `limit` times
__device__ __forceinline__ bool mbar_wait(unsigned mb, unsigned parity, int limit) {
  unsigned ok = 0;
  for (int it = 0; it < limit && !ok; ++it)
    asm volatile(
        "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
        : "=r"(ok)
        : "r"(mb), "r"(parity)
        : "memory");
  return ok != 0;
}

// Shared scratch region, in 8-byte words, used in turn by the condensation
// (stress sums and records of the levels K-1, K-2, ..., two parities), by the
// Newton back-substitution (TF strain increments of two level parities, level
// K: 6G values) and by the strain sums (14 HP words per non-bottom node).
struct Scratch {
  int GX, GY;          // entries of the two condensation parities
  int sx, sy, rx, ry;  // offsets: S sums in HP words, records in TF words from rx
  int words;           // size of the region in 8-byte words
};
__host__ __device__ inline Scratch scratch_layout(int G, int tf_bytes) {
  Scratch c;
  c.GX = G >= 2 ? G / 2 : 1;  // level K-1 has G/2 nodes
  c.GY = G >= 4 ? G / 4 : 1;  // level K-2
  c.sx = 0;
  c.sy = 6 * c.GX;
  const int rx_tf = (6 * c.GX + 6 * c.GY) * (8 / tf_bytes);  // records start after the sums
  c.rx = rx_tf;
  c.ry = rx_tf + ((RS * c.GX + 1) & ~1);
  const int cond_words = (c.ry + RS * c.GY) * tf_bytes / 8 + 1;
  const int chain_words = (9 * G * tf_bytes + 7) / 8;
  const int sum_words = 14 * (G - 1);
  c.words = cond_words;
  if (chain_words > c.words) c.words = chain_words;
  if (sum_words > c.words) c.words = sum_words;
  if (c.words < 64) c.words = 64;  // the epilogue's reduction buffers live here too
  return c;
}
}  // namespace compact_detail
using namespace compact_detail;

// LAW: largest material kind the instance handles (1: thermoelastic and J2;
// 2: also the Perzyna leaf; 3: also the PA66 leaf, whose per-point constants
// (MatPA) follow the materials' and whose leaves keep their history, not
// their internal variables, in zn_s at P.hoff)
template <typename TF, typename HP, int MAXT, int MINB, int LAW>
__global__ void __launch_bounds__(MAXT, MINB) dmn_solve_compact(const SolveParams P) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int K = P.K, N = P.N, G = P.G, ZW = P.zw;
  const int t = threadIdx.x;
  const Scratch sc_ = scratch_layout(G, int(sizeof(TF)));
  HP *a_s = reinterpret_cast<HP *>(smem_raw);  // 3N   jump vectors
  HP *eK = a_s + 3 * N;                        // 6G   strains of the bottom laminates
  HP *zn_s = eK + 6 * G;                       // ZW internal variables at t^n
  HP *eb = zn_s + ZW;                      // 18: eps_bar^{n+1}, deps (HP), eps_bar^{n+1} (FP64)
  double *ebd = reinterpret_cast<double *>(eb + 12);
  HP *sroot = eb + 18;                         // 6: sigma_bar of the last pass
  HP *misc = sroot + 6;                        // 4: 1/dt, D_bar, X_bar
  HP *scr = misc + 4;                          // scratch region (Scratch)
  MatPt<TF, HP> *mp_s = reinterpret_cast<MatPt<TF, HP> *>(scr + sc_.words);
  MatPA<TF, HP> *mpa_s = reinterpret_cast<MatPA<TF, HP> *>(
      (reinterpret_cast<uintptr_t>(mp_s + P.n_mats) + 15) & ~uintptr_t(15));
  Ctrl<TF> *ctrl = reinterpret_cast<Ctrl<TF> *>(
      (reinterpret_cast<uintptr_t>(LAW == 3 ? reinterpret_cast<void *>(mpa_s + P.n_mats)
                                            : reinterpret_cast<void *>(mp_s + P.n_mats)) + 15) &
      ~uintptr_t(15));
  TF *red = reinterpret_cast<TF *>(ctrl + 1);  // 32
  TF *orec = red + 32;                         // 40
  TF *da_s = orec + 40;                        // 3N  Newton increment
  TF *gh_s = da_s + 3 * N;                     // 21N G_p, h_p
  HP *tag = nullptr;
  // condensation: stress sums and records of levels K-1, K-2, ...; level k
  // in X if (K-1-k) is even
  HP *Sx = scr + sc_.sx, *Sy = scr + sc_.sy;
  TF *recX = reinterpret_cast<TF *>(scr) + sc_.rx, *recY = reinterpret_cast<TF *>(scr) + sc_.ry;
  auto recbuf = [&](int k) { return ((K - 1 - k) & 1) ? recY : recX; };
  auto sbuf = [&](int k) { return ((K - 1 - k) & 1) ? Sy : Sx; };
  // back-substitution (the same region): TF strain increments, level k in X
  // if (K - k) is even (level K: G entries of 6)
  TF *tX = reinterpret_cast<TF *>(scr), *tY = tX + 6 * G;
  auto tbuf = [&](int k) { return ((K - k) & 1) ? tY : tX; };
  HP *anc = scr;  // strain sums: per non-bottom node c2 B x, c1 B x, c2 tr, c1 tr
  HP *redD = scr, *redX = scr + 32;  // epilogue: warp sums of D and Diss (32 each)

  const unsigned mask = group_mask(G);
  const int W = group_width(G);
  const int lane = t & 31, warp = t >> 5, nwarp = (G + 31) >> 5;
  if (t == 0) {
    // a warp slot's sub-partition is slot mod 4 and a CTA's warps take
    // consecutive slots: rotate the leader by the CTA's slot group
    unsigned wid;
    asm volatile("mov.u32 %0, %%warpid;" : "=r"(wid));
    ctrl->lead = nwarp > 1 ? int(((wid >> 2) - wid) & unsigned(nwarp - 1)) : 0;
  }
  // mbarrier of the state block's bulk copies (one phase per point)
  __shared__ __align__(8) unsigned long long stage_bar;
  const unsigned mb = smem_u32(&stage_bar);
  unsigned stage_par = 0;
  if (t == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mb) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  const int L = ctrl->lead;
  // node of level k handled by this thread, or -1: a level of more than 32
  // nodes on threads 0.., one of at most 32 nodes on the lanes of warp L
  auto node_at = [&](int k) -> int {
    const int cnt = 1 << (k - 1);
    if (cnt > 32) return t < cnt ? t : -1;
    return (warp == L && lane < cnt) ? lane : -1;
  };
  // the root's record and stress sum, for the decision and the outputs (the
  // layout of the output staging row orec: C, tau at 21, dd at 27, g at 33)
  auto put_root = [&](const Rec<TF> &R, const HP *Sv) {
#pragma unroll
    for (int q = 0; q < 21; ++q) orec[q] = R.C[q];
#pragma unroll
    for (int c = 0; c < 6; ++c) {
      orec[21 + c] = R.tau[c];
      orec[27 + c] = R.dd[c];
      sroot[c] = Sv[c];
    }
    orec[33] = R.gg;
  };

  for (int i = t; i < P.n_mats; i += G)
    mat_static<TF, HP>(mp_s[i], *reinterpret_cast<const MatDev *>(P.mat + kMatWords * i), P.dt);
  if (LAW == 3)
    for (int i = t; i < P.n_mats; i += G)
      if (int(P.mat[kMatWords * i] + 0.5) == 3)
        mat_static_pa<TF, HP>(mpa_s[i], *reinterpret_cast<const MatDev *>(P.mat + kMatWords * i));
  if (t == 0) misc[0] = hp_from(1.0 / P.dt, tag);
  const TF idt_f = TF(1.0 / P.dt);
  const TF tol = TF(P.tol), res_floor = TF(P.res_floor), gamma = TF(P.gamma);

  const HP wL = hp_from(__ldg(P.leafw + 2 * t), tag), wR = hp_from(__ldg(P.leafw + 2 * t + 1), tag);
  int zo0 = P.zoff[2 * t], zo1 = P.zoff[2 * t + 1];
  int zq0 = zo0 >= 0 ? zo0 - (8 + 3 * N) : -1, zq1 = zo1 >= 0 ? zo1 - (8 + 3 * N) : -1;
  int hq0 = LAW == 3 ? P.hoff[2 * t] : zq0, hq1 = LAW == 3 ? P.hoff[2 * t + 1] : zq1;
  int ph0 = P.phase[2 * t], ph1 = P.phase[2 * t + 1];

  // Strains of the bottom laminates by ancestor sums (eq. DMN kinematics):
  // laminate t's strain is the root strain plus, for every ancestor p on its
  // path, +c2 B x_p (the path goes through child 1) or -c1 B x_p (child 2).
  // The two terms of every non-bottom node are formed at once, one node per
  // thread; after one barrier each thread adds its K-1 ancestors' terms root
  // first, the order (and rounding) of a level-by-level top-down sweep.
  //   SW_PLAIN: eK = eps_bar^{n+1} + sum of the B a terms
  //   SW_WARM:  a += da (da_s) on the way; eK as SW_PLAIN at the new a, and
  //             the trace of the strain at (eps_bar^n = tr_root, a^n) of
  //             laminate t is returned (tr B a = a . n)
  //   SW_STEP:  eK += sum of the B da terms (the Newton increment in da_s),
  //             and a += da of the non-bottom nodes on the way
  // Ends with a barrier: eK is complete and the scratch region free again.
  enum { SW_PLAIN = 0, SW_WARM = 1, SW_STEP = 2 };
  auto sweep = [&](int mode, HP tr_root) -> HP {
    for (int q = t; q < G - 1; q += G) {
      const int p = G + q;
      NodeHP<HP> nd;
      load_node(P, p, nd);
      HP x[3];
#pragma unroll
      for (int r = 0; r < 3; ++r) {
        if (mode == SW_STEP) {
          // the step's da of this node: its terms, and a += da (left here by
          // the back-substitution chain, one node per thread)
          const TF d = da_s[3 * p + r];
          x[r] = hp_add_tf(hp_zero(tag), d);
          a_s[3 * p + r] = hp_add_tf(a_s[3 * p + r], d);
        } else {
          x[r] = a_s[3 * p + r];
        }
      }
      HP *ent = anc + 14 * q;
      if (mode == SW_WARM) {
        const HP trj = x[0] * nd.n[0] + x[1] * nd.n[1] + x[2] * nd.n[2];
        ent[12] = nd.c2 * trj;
        ent[13] = nd.c1 * trj;
#pragma unroll
        for (int r = 0; r < 3; ++r) {
          x[r] = hp_add_tf(x[r], da_s[3 * p + r]);
          a_s[3 * p + r] = x[r];
        }
      }
      HP J[6];
      bvec_hp(nd, x, J);
#pragma unroll
      for (int c = 0; c < 6; ++c) {
        ent[c] = nd.c2 * J[c];
        ent[6 + c] = nd.c1 * J[c];
      }
    }
    __syncthreads();
    HP e[6], tr = tr_root;
#pragma unroll
    for (int c = 0; c < 6; ++c) e[c] = mode == SW_STEP ? hp_zero(tag) : eb[c];
    for (int k = 1; k <= K - 1; ++k) {
      const int p = (1 << K) - (1 << k) + (t >> (K - k));
      const HP *ent = anc + 14 * (p - G);
      if ((t >> (K - k - 1)) & 1) {
#pragma unroll
        for (int c = 0; c < 6; ++c) e[c] = e[c] - ent[6 + c];
        if (mode == SW_WARM) tr = tr - ent[13];
      } else {
#pragma unroll
        for (int c = 0; c < 6; ++c) e[c] = e[c] + ent[c];
        if (mode == SW_WARM) tr = tr + ent[12];
      }
    }
#pragma unroll
    for (int c = 0; c < 6; ++c) eK[6 * t + c] = mode == SW_STEP ? eK[6 * t + c] + e[c] : e[c];
    __syncthreads();
    return tr;
  };

  for (;;) {
    if (t == 0) {
      unsigned long long q = atomicAdd(P.queue, 1ull);
      while (P.skip && q < (unsigned long long)P.n_points && P.skip[q] != 0) q = atomicAdd(P.queue, 1ull);
      ctrl->next = q;
    }
    __syncthreads();
    const int64_t pt = int64_t(ctrl->next);
    if (pt >= P.n_points) break;
    DMN_BOUNDS_CLEAR();
#ifdef DMN_BOUNDS_CHECK
    check_leaf(P, mp_s, ph0, hq0, zq0, ZW);
    check_leaf(P, mp_s, ph1, hq1, zq1, ZW);
    zo0 = zq0 >= 0 ? zq0 + 8 + 3 * N : -1;
    zo1 = zq1 >= 0 ? zq1 + 8 + 3 * N : -1;
#endif
    const double *sin = P.sin + pt * P.SW;
    double *sout = P.sout + pt * P.SW;
    HP *zw = reinterpret_cast<HP *>(sout + 8 + 3 * N);  // z of the current pass (8-byte slots)
    const double theta = P.theta[pt];
    {
      // the state block by bulk copies (a, and z unless LAW 3 keeps histories
      // there), or by plain loads where the caller's state is not 16-byte
      // aligned; with them the predicted increment, eps_bar^n and deps
      constexpr int U = 8;
      const bool bulk = (reinterpret_cast<uintptr_t>(P.sin) & 15) == 0;
      if (bulk && t == 0) {
        const unsigned n1 = unsigned(3 * N + 1) * 8u, n2 = LAW < 3 ? unsigned((ZW + 2) & ~1) * 8u : 0u;
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mb), "r"(n1 + n2) : "memory");
        bulk_g2s(smem_u32(a_s), sin + 8, n1, mb);
        if (LAW < 3) bulk_g2s(smem_u32(zn_s - 1), sin + 7 + 3 * N, n2, mb);
      }
      double ve = 0.0, vd = 0.0;
      float vp[U];
      const float *d0 = P.da0 ? P.da0 + pt * (3 * N) : nullptr;
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int i = t + u * G;
        vp[u] = d0 && i < 3 * N ? ld_stream(d0 + i) : 0.0f;
      }
      if (G >= 8 && t < 6) {
        ve = ld_stream(sin + t);
        vd = ld_stream(P.deps + pt * 6 + t);
      }
      if (d0) {
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int i = t + u * G;
          if (i < 3 * N) da_s[i] = TF(vp[u]);
        }
      }
      if (bulk) {
        const bool ok = mbar_wait(mb, stage_par, kWaitLimit);
        if (!__syncthreads_and(ok)) {
          // the copies did not complete: flag the point, give them time to
          // land, and stop this CTA (the queue hands its points to the others)
          mbar_wait(mb, stage_par, kWaitLimit);
          if (t == 0) {
            P.status[pt] = kPtStaging;
            P.iters[pt] = 0;
          }
          return;
        }
        stage_par ^= 1u;
        if (sizeof(TF) == 4) {  // mixed: the raw FP64 words into float-float, in place
          const double *ra = reinterpret_cast<const double *>(a_s);
          const double *rz = reinterpret_cast<const double *>(zn_s);
#pragma unroll 1
          for (int i = t; i < 3 * N; i += G) a_s[i] = hp_load(ra[i], tag);
          if (LAW < 3) {
#pragma unroll 1
            for (int i = t; i < ZW; i += G) zn_s[i] = hp_load(rz[i], tag);
          }
        }
      } else {
#pragma unroll 1
        for (int i = t; i < 3 * N; i += G) a_s[i] = hp_load(ld_stream(sin + 8 + i), tag);
        if (LAW < 3) {
#pragma unroll 1
          for (int i = t; i < ZW; i += G) zn_s[i] = hp_load(ld_stream(sin + 8 + 3 * N + i), tag);
        }
      }
      if (G >= 8) {
        if (t < 6) {
          ebd[t] = ve + vd;  // eps_bar^{n+1} = eps_bar^n + deps exactly in FP64
          eb[t] = hp_load(ve + vd, tag);
          eb[6 + t] = hp_load(vd, tag);
        }
      } else {
        for (int c = t; c < 6; c += G) {
          const double d = P.deps[pt * 6 + c], e1 = sin[c] + d;
          ebd[c] = e1;
          eb[c] = hp_load(e1, tag);
          eb[6 + c] = hp_load(d, tag);
        }
      }
    }
    __syncthreads();
    for (int i = t; i < P.n_mats; i += G) mat_point<TF, HP, LAW>(mp_s[i], hp_load(theta, tag), misc[0], idt_f);
    if (LAW == 3) {
      // PA66 constants at this temperature, then each thread's leaves: the
      // history of a PA66 leaf, the internal variables of a J2 leaf
      for (int i = t; i < P.n_mats; i += G)
        if (mp_s[i].kind == 3)
          mat_point_pa<TF, HP>(mpa_s[i], *reinterpret_cast<const MatDev *>(P.mat + kMatWords * i), theta,
                               P.dt);
      __syncthreads();
#pragma unroll 1
      for (int sd = 0; sd < 2; ++sd) {
        const int j = 2 * t + sd, zo = sd ? zo1 : zo0, ph = sd ? ph1 : ph0, hq = sd ? hq1 : hq0;
        if (zo < 0) continue;
        if (mp_s[ph].kind == 3) {
          pa_history<TF, HP>(mpa_s[ph], sin + zo, zn_s + hq);
        } else {
          const int nz = mp_s[ph].kind == 1 ? 7 : 13;
          for (int c = 0; c < nz; ++c) zn_s[hq + c] = hp_load(sin[zo + c], tag);
        }
        (void)j;
      }
    }
    if (t == 0) {
      ctrl->first = 1;
      ctrl->it = 0;
      ctrl->bt = 0;
      ctrl->gi = TF(1);
      ctrl->res_old = TF(0);
      ctrl->status = 0;
    }
    const HP *zn0 = hq0 >= 0 ? zn_s + hq0 : nullptr;
    const HP *zn1 = hq1 >= 0 ? zn_s + hq1 : nullptr;
    HP *zw0 = zq0 >= 0 ? zw + zq0 : nullptr;
    HP *zw1 = zq1 >= 0 ? zw + zq1 : nullptr;

    HP trn0 = hp_zero(tag), trn1 = hp_zero(tag);
    bool first = true;  // the first pass also yields the traces of eps^n
    if (P.da0) {
      // warm start a^n + da0; the traces of eps^n come with the same sweep
      const HP tre =
          sweep(SW_WARM, hp_load(sin[0], tag) + hp_load(sin[1], tag) + hp_load(sin[2], tag));
      NodeHP<HP> nd;
      load_node(P, t, nd);
      const HP an[3] = {a_s[3 * t], a_s[3 * t + 1], a_s[3 * t + 2]};  // still a^n
      const HP trj = an[0] * nd.n[0] + an[1] * nd.n[1] + an[2] * nd.n[2];
      trn0 = tre + nd.c2 * trj;
      trn1 = tre - nd.c1 * trj;
#pragma unroll
      for (int r = 0; r < 3; ++r) a_s[3 * t + r] = hp_add_tf(an[r], da_s[3 * t + r]);
      first = false;  // thread t alone uses a_s[3t..] until the next barrier
    } else {
      sweep(SW_PLAIN, hp_zero(tag));  // strains of the bottom laminates at a^n
    }
    int attempt = 0, it_total = 0;
    HP Dsum = hp_zero(tag), Xsum = hp_zero(tag);
    Rec<TF> rec;
    for (;;) {
      // Algorithm 1 takes at least one Newton step (maxit >= 1), so the
      // first pass of an iteration never gives the outputs: it skips their
      // terms (coupling term, dissipation, thermal tangents)
      const bool full = !ctrl->first;
      // ---- R2: leaves and laminate t ----
      TF r2;
      HP S[6];
      {
        NodeHP<HP> nd;
        load_node(P, t, nd);
        HP el[6], er[6];
        {
          const HP av[3] = {a_s[3 * t], a_s[3 * t + 1], a_s[3 * t + 2]};
          HP J[6];
          bvec_hp(nd, av, J);
#pragma unroll
          for (int c = 0; c < 6; ++c) {
            const HP e = eK[6 * t + c];
            el[c] = e + nd.c2 * J[c];
            er[c] = e - nd.c1 * J[c];
          }
        }
        if (first) {  // at a = a^n: eps^n = eps - deps
          const HP trd = eb[6] + eb[7] + eb[8];
          trn0 = (el[0] + el[1] + el[2]) - trd;
          trn1 = (er[0] + er[1] + er[2]) - trd;
        }
        HP sl[6], sr[6], DL, DR, XL, XR;
        Rec<TF> rr;
        if (LAW == 3 && mp_s[ph0].kind == 3)
          leaf_pa66<TF, HP>(mp_s[ph0], mpa_s[ph0], el, zn0, trn0, sl, DL, XL, rec, zw0);
        else
          leaf_eval<TF, HP, LAW>(mp_s[ph0], el, zn0, trn0, sl, DL, XL, rec, zw0, full);
        if (LAW == 3 && mp_s[ph1].kind == 3)
          leaf_pa66<TF, HP>(mp_s[ph1], mpa_s[ph1], er, zn1, trn1, sr, DR, XR, rr, zw1);
        else
          leaf_eval<TF, HP, LAW>(mp_s[ph1], er, zn1, trn1, sr, DR, XR, rr, zw1, full);
        if (full) {
          Dsum = wL * DL + wR * DR;
          Xsum = wL * XL + wR * XR;
        }
        HP dsh[6];
#pragma unroll
        for (int c = 0; c < 6; ++c) {
          S[c] = wL * sl[c] + wR * sr[c];
          dsh[c] = sl[c] - sr[c];
        }
        HP rbh[3];
        btvec_hp(nd, dsh, rbh);  // B^T (sigma_L - sigma_R) = r_t / (w c1 c2)
        TF n[3], c1, c2, iwcc, wcc;
        load_node_tf(P, t, n, c1, c2, iwcc, wcc);
        const TF rbv[3] = {tf_of(rbh[0], (TF *)nullptr), tf_of(rbh[1], (TF *)nullptr),
                           tf_of(rbh[2], (TF *)nullptr)};
        r2 = wcc * wcc * (rbv[0] * rbv[0] + rbv[1] * rbv[1] + rbv[2] * rbv[2]);
        combine<TF>(rec, rr, n, c1, c2, rbv, gh_s + 21 * t, full);
        if (K == 1) put_root(rec, S);
      }
      // ---- level K-1: neighbouring lanes (2j, 2j+1) ----
      if (K >= 2) {
        Rec<TF> other;
        rec_shfl_down(other, rec, 1, mask, W);
        HP So[6];
#pragma unroll
        for (int c = 0; c < 6; ++c) So[c] = hp_shfl_down(mask, S[c], 1, W);
        if ((t & 1) == 0) {
          const int j = t >> 1;
          const int p = (1 << K) - (1 << (K - 1)) + j;
          NodeHP<HP> nd;
          load_node(P, p, nd);
          HP dh[6];
#pragma unroll
          for (int c = 0; c < 6; ++c) {
            dh[c] = nd.c2 * S[c] - nd.c1 * So[c];
            S[c] = S[c] + So[c];
          }
          HP rh[3];
          btvec_hp(nd, dh, rh);  // r_p = B^T (c2 S_L - c1 S_R)
          TF n[3], c1, c2, iwcc, wcc;
          load_node_tf(P, p, n, c1, c2, iwcc, wcc);
          const TF rv[3] = {tf_of(rh[0], (TF *)nullptr), tf_of(rh[1], (TF *)nullptr),
                            tf_of(rh[2], (TF *)nullptr)};
          r2 += rv[0] * rv[0] + rv[1] * rv[1] + rv[2] * rv[2];
          const TF rbv[3] = {rv[0] * iwcc, rv[1] * iwcc, rv[2] * iwcc};
          combine<TF>(rec, other, n, c1, c2, rbv, gh_s + 21 * p, full);
          if (K >= 3) {
            rec_put(recX + RS * j, rec);
#pragma unroll
            for (int c = 0; c < 6; ++c) Sx[6 * j + c] = S[c];
          } else {
            put_root(rec, S);
          }
        }
      }
      // ---- levels K-2 .. 1, by Mandel rows: node j of level k on the
      //      eight lanes 8j .. 8j + 7 of the level's tasks (combine_rows).  A
      //      level of more than 32 tasks runs on all threads between block
      //      barriers; once the producers of the level below all sit in warp
      //      L, warp L goes on alone with warp barriers and the other warps
      //      move to the reduction barrier.  A CTA of fewer than 8 threads
      //      (K = 3) condenses its root on one thread. ----
      if (G >= 8) {
        for (int k = K - 2; k >= 1; --k) {
          const int ntask = 8 << (k - 1);
          const bool wide = ntask > 32 && G > 32;
          const bool prod_wide = k + 1 == K - 1 ? G > 32 : (2 * ntask > 32 && G > 32);
          if (prod_wide) __syncthreads();
          if (!wide) {  // this level and the ones above: warp L alone
            if (warp != L) break;
            if (!prod_wide) __syncwarp(mask);
          }
          const int step = wide ? G : (G < 32 ? G : 32);
          const int q0 = wide ? t : lane;
          const int cnt = 1 << (k - 1);
          for (int qb = 0; qb < ntask; qb += step) {
            if (qb + (q0 & ~31) >= ntask) break;  // the whole warp is past the level
            const int q = qb + q0;
            const bool st = q < ntask;            // else a copy of the last node, not stored
            const int j = st ? q >> 3 : cnt - 1;
            const int p = (1 << K) - (1 << k) + j;
            // children: slots 2j, 2j + 1 of level k + 1's buffer (debug build: checked)
            const int cap = ((K - 1 - (k + 1)) & 1) ? sc_.GY : sc_.GX;
            const int jc = DMN_IDX(2 * j, cap - 1) >> 1;
            (void)cap;
            const TF *rc = recbuf(k + 1) + RS * (2 * jc);
            const HP *sc = sbuf(k + 1) + 12 * jc;
            TF *dst = orec;
            HP *sd = sroot;
            if (k > 1) {
              const int js = DMN_IDX(j, ((K - 1 - k) & 1) ? sc_.GY : sc_.GX);
              dst = recbuf(k) + RS * js;
              sd = sbuf(k) + 6 * js;
            }
            combine_rows<TF, HP>(P, p, q & 7, st, mask, rc, rc + RS, sc, sc + 6, dst, sd, gh_s + 21 * p, r2,
                                 full, k == 1);
          }
        }
      } else if (K == 3) {
        __syncwarp(mask);
        if (t == 0) {
          const int p = (1 << K) - 2;
          const TF *rc = recX;
          const HP *sc = Sx;
          Rec<TF> other;
          rec_get(rec, rc);
          rec_get(other, rc + RS);
          NodeHP<HP> nd;
          load_node(P, p, nd);
          HP dh[6];
#pragma unroll
          for (int c = 0; c < 6; ++c) {
            const HP SL = sc[c], SR = sc[6 + c];
            S[c] = SL + SR;
            dh[c] = nd.c2 * SL - nd.c1 * SR;
          }
          HP rh[3];
          btvec_hp(nd, dh, rh);
          TF n[3], c1, c2, iwcc, wcc;
          load_node_tf(P, p, n, c1, c2, iwcc, wcc);
          const TF rv[3] = {tf_of(rh[0], (TF *)nullptr), tf_of(rh[1], (TF *)nullptr),
                            tf_of(rh[2], (TF *)nullptr)};
          r2 += rv[0] * rv[0] + rv[1] * rv[1] + rv[2] * rv[2];
          const TF rbv[3] = {rv[0] * iwcc, rv[1] * iwcc, rv[2] * iwcc};
          combine<TF>(rec, other, n, c1, c2, rbv, gh_s + 21 * p, full);
          put_root(rec, S);
        }
      }
      // ---- residual norm, decision (Algorithm 1) ----
      r2 = warp_sum(r2, mask, W);
      if (lane == 0) red[warp] = r2;
      __syncthreads();
      if (t == 0) {
        TF s = TF(0);
        for (int w = 0; w < nwarp; ++w) s += red[w];
        TF sn = TF(0);
#pragma unroll
        for (int c = 0; c < 6; ++c) {
          const TF v = tf_of(sroot[c], (TF *)nullptr);
          sn += v * v;
        }
        TF den = sqrt(sn);
        if (den < res_floor) den = res_floor;
        const TF res = sqrt(s) / (TF(N) * den);
        Ctrl<TF> &c = *ctrl;
        const bool accept = c.first || (res < c.res_old) || (c.bt >= P.maxbt);
        int action;
        if (accept) {
          if (!isfinite(res)) {
            c.status = 2;
            action = ACT_DONE;
          } else if (!c.first && res < tol) {
            c.status = 0;
            action = ACT_DONE;
          } else if (c.it >= P.maxit) {
            c.status = 1;
            action = ACT_DONE;
          } else {
            c.res_old = res;
            c.it += 1;
            c.bt = 0;
            c.gi = TF(1);
            action = ACT_STEP;
          }
          c.first = 0;
        } else {
          action = ACT_BACK;
        }
        c.res = res;
        c.action = action;
      }
      first = false;
      __syncthreads();
      const int action = ctrl->action;
      if (action == ACT_DONE) {
        if (P.da0 && attempt == 0 && ctrl->status != 0) {
          // warm-started iteration failed: run Algorithm 1 again from a^n
          attempt = 1;
          it_total = ctrl->it;
          for (int i = t; i < 3 * N; i += G) a_s[i] = hp_load(sin[8 + i], tag);
          __syncthreads();  // every thread has read ctrl->status and ctrl->it
          if (t == 0) {
            ctrl->first = 1;
            ctrl->it = 0;
            ctrl->bt = 0;
            ctrl->gi = TF(1);
            ctrl->res_old = TF(0);
            ctrl->status = 0;
          }
          sweep(SW_PLAIN, hp_zero(tag));  // its barriers order the reset before later reads
          continue;
        }
        break;
      }
      if (action == ACT_STEP) {
        // ---- back-substitution in TF, node j of level k on one thread:
        //      da_p = -(G_p de_p + h_p); children de + c2 B da, de - c1 B da;
        //      then the bottom strains take the high-precision sum of the
        //      B da terms of their ancestors
        for (int k = 1; k <= K; ++k) {
          const int j = node_at(k);  // level K: j = t
          if (j >= 0) {
            const int p = DMN_IDX((1 << K) - (1 << k) + j, N);
            TF de[6];
            if (k == 1) {
#pragma unroll
              for (int c = 0; c < 6; ++c) de[c] = TF(0);
            } else {
              const TF *src = tbuf(k) + DMN_IDX(6 * j, 6 * G - 5);
#pragma unroll
              for (int c = 0; c < 6; ++c) de[c] = src[c];
            }
            const TF *g = gh_s + 21 * p;
            TF da[3];
#pragma unroll
            for (int r = 0; r < 3; ++r) {
              TF sum = g[18 + r];
#pragma unroll
              for (int c = 0; c < 6; ++c) sum += g[6 * r + c] * de[c];
              da[r] = -sum;
            }
#pragma unroll
            for (int r = 0; r < 3; ++r) da_s[3 * p + r] = da[r];
            if (k == K) {  // the other levels' a += da: in the strain sums that follow
#pragma unroll
              for (int r = 0; r < 3; ++r) a_s[3 * p + r] = hp_add_tf(a_s[3 * p + r], da[r]);
            }
            if (k < K) {
              TF n[3], c1, c2, iwcc, wcc;
              load_node_tf(P, p, n, c1, c2, iwcc, wcc);
              TF J[6];
              bvec(n, da, J);
              TF *dst = tbuf(k + 1) + DMN_IDX(12 * j, 6 * G - 11);
#pragma unroll
              for (int c = 0; c < 6; ++c) {
                dst[c] = de[c] + c2 * J[c];
                dst[6 + c] = de[c] - c1 * J[c];
              }
            }
          }
          // level k+1 is read by threads < 2^k: a warp barrier while they
          // all sit in warp L (the other warps wait at the next block barrier)
          if (k == K || (1 << k) > 32) __syncthreads();
          else if (warp == L) __syncwarp(mask);
        }
        sweep(SW_STEP, hp_zero(tag));
      } else {
        // ---- backtracking (rare): a -= f da, strains from a new sweep ----
        const TF f = ctrl->gi * (TF(1) - gamma);
        for (int i = t; i < 3 * N; i += G) a_s[i] = hp_add_tf(a_s[i], -f * da_s[i]);
        __syncthreads();
        sweep(SW_PLAIN, hp_zero(tag));  // its barriers also order the reads of ctrl->gi above
        if (t == 0) {
          ctrl->gi *= gamma;
          ctrl->bt += 1;
        }
      }
    }

    // ---- outputs and state (the last pass is at the final a; its coupling
    //      term and dissipation sums are still in the registers) ----
    {
      const HP ds_ = warp_sum(Dsum, mask, W), xs_ = warp_sum(Xsum, mask, W);
      if (lane == 0) {
        redD[warp] = ds_;
        redX[warp] = xs_;
      }
    }
    __syncthreads();
    if (t == 0) {
      HP Db = redD[0], Xb = redX[0];
      for (int w = 1; w < nwarp; ++w) {
        Db = Db + redD[w];
        Xb = Xb + redX[w];
      }
      misc[1] = Db;
      misc[2] = Xb;
    }
    __syncthreads();
    int bad = 0;
    for (int c = t; c < kOutWords; c += G) {
      double v;
      if (c < 6) v = hp_to(sroot[c]);
      else if (c < 42) v = double(sget(orec, (c - 6) / 6, (c - 6) % 6));
      else if (c < 48) v = double(orec[21 + c - 42]);
      else if (c == 48) v = hp_to(misc[1]);
      else if (c < 55) v = double(orec[27 + c - 49]);
      else if (c == 55) v = double(orec[33]);
      else v = hp_to(misc[2]);
      if (!isfinite(v)) bad = 1;
      __stcs(P.out + pt * kOutWords + c, v);
    }
    bad = __syncthreads_or(bad);
    const int bbad = DMN_BOUNDS_CTA_OR();
    if (t == 0) {
      P.status[pt] = (bad ? 2 : ctrl->status) | (attempt ? 4 : 0) | (bbad ? kPtBounds : 0);
      P.iters[pt] = ctrl->it + it_total;
    }
    for (int c = t; c < 8; c += G) sout[c] = c < 6 ? ebd[c] : (c == 6 ? theta : 0.0);
    for (int i = t; i < 3 * N; i += G) __stcs(sout + 8 + i, hp_to(a_s[i]));
    if (LAW == 3) {  // each thread its own leaves (it parked their values itself)
#pragma unroll 1
      for (int sd = 0; sd < 2; ++sd) {
        const int zo = sd ? zo1 : zo0, ph = sd ? ph1 : ph0;
        if (zo < 0) continue;
        if (mp_s[ph].kind == 3) {
          pa_finish<TF, HP>(mpa_s[ph], sin + zo, sout + zo);
        } else {
          const int nz = mp_s[ph].kind == 1 ? 7 : 13;
          const HP *zp = reinterpret_cast<const HP *>(sout + zo);
          for (int c = 0; c < nz; ++c) {
            const HP v = zp[c];
            sout[zo + c] = hp_to(v);
          }
        }
      }
    } else {
      for (int i0 = t; i0 < ZW; i0 += 8 * G) {  // parked internal variables -> FP64 in place
        HP v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) v[u] = i0 + u * G < ZW ? ld_once(zw + i0 + u * G) : hp_zero(tag);
#pragma unroll
        for (int u = 0; u < 8; ++u)
          if (i0 + u * G < ZW) __stcs(sout + 8 + 3 * N + i0 + u * G, hp_to(v[u]));
      }
    }
    for (int i = P.zend + t; i < P.SW; i += G) sout[i] = 0.0;  // padding word
    __syncthreads();
  }
}

}  // namespace dmn
