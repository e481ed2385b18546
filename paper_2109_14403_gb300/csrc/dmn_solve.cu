// dmn_solve.cu -- the Newton solve of Algorithm 1 (arXiv 2109.14403, Sec. 3.3)
// for one Gauss point per CTA.  See dmn_kernels.cuh for the mapping and the
// condensation.
#include "dmn_internal.h"
#include "solve_common.cuh"

namespace dmn {

// Top-down back-substitution of the Newton increment (owner mapping):
// da_p = -(G_p de_p + h_p); children de_1 = de + c2 B da, de_2 = de - c1 B da.
template <typename TF>
__device__ __forceinline__ void back_substitute(const SolveParams &P, TF *da_s, const TF *gh_s,
                                                double *xslot, int t) {
  const int K = P.K;
  const unsigned mask = group_mask(P.G);
  const int W = group_width(P.G);
  TF e[6] = {TF(0), TF(0), TF(0), TF(0), TF(0), TF(0)};
  for (int k = 1; k <= K; ++k) {
    const int span = 1 << (K - k);
    const int off = span >> 1;
    const bool owner = (t & (span - 1)) == 0;
    TF c2e[6] = {TF(0), TF(0), TF(0), TF(0), TF(0), TF(0)};
    if (owner) {
      const int p = (1 << K) - (1 << k) + (t >> (K - k));
      const TF *g = gh_s + 21 * p;
      TF da[3];
#pragma unroll
      for (int r = 0; r < 3; ++r) {
        TF s = g[18 + r];
#pragma unroll
        for (int c = 0; c < 6; ++c) s += g[6 * r + c] * e[c];
        da[r] = -s;
      }
#pragma unroll
      for (int r = 0; r < 3; ++r) da_s[3 * p + r] = da[r];
      if (k < K) {
        TF n[3], c1, c2, iw, w;
        load_node_tf(P, p, n, c1, c2, iw, w);
        TF ba[6];
        bvec(n, da, ba);
#pragma unroll
        for (int c = 0; c < 6; ++c) {
          c2e[c] = e[c] - c1 * ba[c];
          e[c] = e[c] + c2 * ba[c];
        }
      }
    }
    if (k == K) break;
    if (off >= 32) {
      if (owner) {
#pragma unroll
        for (int c = 0; c < 6; ++c) xslot[6 * (t / span) + c] = double(c2e[c]);
      }
      __syncthreads();
      if ((t & (span - 1)) == off) {
#pragma unroll
        for (int c = 0; c < 6; ++c) e[c] = TF(xslot[6 * ((t - off) / span) + c]);
      }
      __syncthreads();
    } else {
      const bool recv = (t & (span - 1)) == off;
#pragma unroll
      for (int c = 0; c < 6; ++c) {
        const TF v = __shfl_up_sync(mask, c2e[c], off, W);
        if (recv) e[c] = v;
      }
    }
  }
}

// One Newton pass ("Residual" of Algorithm 1 plus the condensation):
//  R1  compact top-down strain scatter in HP: node j of level k on thread j;
//  R2  thread t: leaves 2t, 2t+1 (HP stress, TF record) and laminate t;
//  R3  per level, bottom-up: compact HP subtree stress sums S and residual
//      r_p = B^T (c2 S_L - c1 S_R), then the owner-mapped TF condensation.
// HP = double (FP64 path) or float-float (mixed path); TF = double or float.
// MAXT bounds the threads per CTA (2^(K-1)); MINB asks the compiler to fit
// MINB CTAs per SM (register budget 65536 / (MAXT * MINB)).  Points are taken
// from a device-side queue (one atomic counter per launch), so a CTA whose
// point converged moves on at once: uneven Newton iteration counts do not
// leave CTAs idle.
template <typename TF, typename HP, int MAXT, int MINB>
__global__ void __launch_bounds__(MAXT, MINB) dmn_solve_kernel(const SolveParams P) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int K = P.K, N = P.N, G = P.G, ZW = P.zw;
  const int t = threadIdx.x;
  const int nslot = G >= 64 ? G / 64 : 1;
  HP *a_s = reinterpret_cast<HP *>(smem_raw);  // 3N   jump vectors
  // node strains (top-down) and subtree stress sums (bottom-up) of two
  // consecutive levels: level k lives in the buffer of its parity
  HP *esK = a_s + 3 * N;                       // 6G   levels K, K-2, ...
  HP *esO = esK + 6 * G;                       // 3G   levels K-1, K-3, ...
  HP *zn_s = esO + 3 * G;                      // ZW internal variables at t^n
  HP *zw_s = zn_s + ZW;                        // ZW internal variables of the last pass
  HP *eb = zw_s + ZW;                          // 12: eps_bar^{n+1}, deps
  HP *redD = eb + 12;                          // 32
  HP *redX = redD + 32;                        // 32
  HP *misc = redX + 32;                        // 4: 1/dt, D_bar, X_bar
  double *slots = reinterpret_cast<double *>(misc + 4);  // nslot * kRecWords
  MatPt<TF, HP> *mp_s = reinterpret_cast<MatPt<TF, HP> *>(slots + nslot * kRecWords);
  Ctrl<TF> *ctrl = reinterpret_cast<Ctrl<TF> *>(mp_s + P.n_mats);
  TF *red = reinterpret_cast<TF *>(ctrl + 1);   // 32  warp partial sums of |r|^2
  TF *orec = red + 32;                          // 40  root record for the outputs
  TF *da_s = orec + 40;                         // 3N  Newton increment
  TF *gh_s = da_s + 3 * N;                      // 21N G_p, h_p
  TF *rb_s = gh_s + 21 * N;                     // 3 max(1, G/2): residual / (w c1 c2), one level
  HP *tag = nullptr;

  const unsigned mask = group_mask(G);
  const int W = group_width(G);
  const int lane = t & 31, warp = t >> 5, nwarp = (G + 31) >> 5;
  auto lev = [&](int k) { return ((k ^ K) & 1) ? esO : esK; };  // buffer of level k
  HP *const es1 = lev(1);  // root: strain, then sigma_bar
  // top-down strain scatter from the root strain (eq. DMN kinematics): node j
  // of level k on thread j; on return esK holds the bottom laminates' strains
  auto scatter = [&](const HP *root) {
    for (int c = t; c < 6; c += G) es1[c] = root[c];
    __syncthreads();
    for (int k = 1; k <= K - 1; ++k) {
      if (t < (1 << (k - 1))) {
        const int p = (1 << K) - (1 << k) + t;
        HP *ep = lev(k) + 6 * t, *ec = lev(k + 1) + 12 * t;
        NodeHP<HP> nd;
        load_node(P, p, nd);
        const HP av[3] = {a_s[3 * p], a_s[3 * p + 1], a_s[3 * p + 2]};
        HP J[6];
        bvec_hp(nd, av, J);
#pragma unroll
        for (int c = 0; c < 6; ++c) {
          const HP e = ep[c];
          ec[c] = e + nd.c2 * J[c];
          ec[6 + c] = e - nd.c1 * J[c];
        }
      }
      __syncthreads();
    }
  };

  for (int i = t; i < P.n_mats; i += G)
    mat_static<TF, HP>(mp_s[i], *reinterpret_cast<const MatDev *>(P.mat + kMatWords * i), P.dt);
  if (t == 0) misc[0] = hp_from(1.0 / P.dt, tag);
  const TF idt_f = TF(1.0 / P.dt);
  const TF tol = TF(P.tol), res_floor = TF(P.res_floor), gamma = TF(P.gamma);

  // per-thread constants: laminate t and its leaves 2t, 2t+1
  const HP wL = hp_from(__ldg(P.leafw + 2 * t), tag), wR = hp_from(__ldg(P.leafw + 2 * t + 1), tag);
  const int zo0 = P.zoff[2 * t], zo1 = P.zoff[2 * t + 1];
  int zq0 = zo0 >= 0 ? zo0 - (8 + 3 * N) : -1, zq1 = zo1 >= 0 ? zo1 - (8 + 3 * N) : -1;
  int ph0 = P.phase[2 * t], ph1 = P.phase[2 * t + 1];

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
    {
      int hq0 = zq0, hq1 = zq1;  // the shared copy of z uses the state's offsets
      check_leaf(P, mp_s, ph0, hq0, zq0, ZW);
      check_leaf(P, mp_s, ph1, hq1, zq1, ZW);
    }
#endif
    const double *sin = P.sin + pt * P.SW;
    double *sout = P.sout + pt * P.SW;
    const double theta = P.theta[pt];
    for (int i = t; i < 3 * N; i += G) a_s[i] = hp_load(sin[8 + i], tag);
    for (int i = t; i < ZW; i += G) zn_s[i] = hp_load(sin[8 + 3 * N + i], tag);
    for (int c = t; c < 6; c += G) {  // a point may have fewer than 6 threads
      const double d = P.deps[pt * 6 + c];
      eb[c] = hp_load(sin[c] + d, tag);
      eb[6 + c] = hp_load(d, tag);
    }
    __syncthreads();  // misc[0] (first point) and the static material part
    for (int i = t; i < P.n_mats; i += G) mat_point<TF, HP, 1>(mp_s[i], hp_load(theta, tag), misc[0], idt_f);
    if (t == 0) {
      ctrl->first = 1;
      ctrl->it = 0;
      ctrl->bt = 0;
      ctrl->gi = TF(1);
      ctrl->res_old = TF(0);
      ctrl->status = 0;
    }
    __syncthreads();
    const HP *zn0 = zq0 >= 0 ? zn_s + zq0 : nullptr;
    const HP *zn1 = zq1 >= 0 ? zn_s + zq1 : nullptr;
    HP *zw0 = zq0 >= 0 ? zw_s + zq0 : nullptr;
    HP *zw1 = zq1 >= 0 ? zw_s + zq1 : nullptr;

    HP trn0 = hp_zero(tag), trn1 = hp_zero(tag);
    bool first = true;  // the first pass also yields the traces of eps^n
    if (P.da0) {
      // warm start a^n + da0: the traces of eps^n come from a scatter at a^n
      HP ebn[6];
      for (int c = 0; c < 6; ++c) ebn[c] = hp_load(sin[c], tag);  // eps_bar^n
      __syncthreads();
      scatter(ebn);
      NodeHP<HP> nd;
      load_node(P, t, nd);
      const HP av[3] = {a_s[3 * t], a_s[3 * t + 1], a_s[3 * t + 2]};
      HP J[6];
      bvec_hp(nd, av, J);
      const HP trj = J[0] + J[1] + J[2];
      const HP tre = esK[6 * t] + esK[6 * t + 1] + esK[6 * t + 2];
      trn0 = tre + nd.c2 * trj;
      trn1 = tre - nd.c1 * trj;
      first = false;
      __syncthreads();
      const float *d0 = P.da0 + pt * (3 * N);
      for (int i = t; i < 3 * N; i += G) a_s[i] = hp_add_tf(a_s[i], TF(d0[i]));
      __syncthreads();
    }
    int attempt = 0, it_total = 0;
    HP Dsum = hp_zero(tag), Xsum = hp_zero(tag);
    Rec<TF> rec;
    for (;;) {
      // ---- R1: strains, top-down (eq. DMN kinematics) ----
      scatter(eb);
      // ---- R2: leaves and laminate t ----
      TF r2;
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
            const HP e = esK[6 * t + c];
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
        leaf_eval<TF, HP, 1>(mp_s[ph0], el, zn0, trn0, sl, DL, XL, rec, zw0);
        leaf_eval<TF, HP, 1>(mp_s[ph1], er, zn1, trn1, sr, DR, XR, rr, zw1);
        Dsum = wL * DL + wR * DR;
        Xsum = wL * XL + wR * XR;
        HP dsh[6];
#pragma unroll
        for (int c = 0; c < 6; ++c) {
          esK[6 * t + c] = wL * sl[c] + wR * sr[c];
          dsh[c] = sl[c] - sr[c];
        }
        HP rbh[3];
        btvec_hp(nd, dsh, rbh);  // B^T (sigma_L - sigma_R) = r_t / (w c1 c2)
        TF n[3], c1, c2, iwcc, wcc;
        load_node_tf(P, t, n, c1, c2, iwcc, wcc);
        const TF rbv[3] = {tf_of(rbh[0], (TF *)nullptr), tf_of(rbh[1], (TF *)nullptr),
                           tf_of(rbh[2], (TF *)nullptr)};
        r2 = wcc * wcc * (rbv[0] * rbv[0] + rbv[1] * rbv[1] + rbv[2] * rbv[2]);
        combine<TF>(rec, rr, n, c1, c2, rbv, gh_s + 21 * t);
      }
      // ---- R3: bottom-up ----
      for (int k = K - 1; k >= 1; --k) {
        __syncthreads();
        if (t < (1 << (k - 1))) {
          const int p = (1 << K) - (1 << k) + t;
          HP *sp = lev(k) + 6 * t;
          const HP *sc = lev(k + 1) + 12 * t;
          NodeHP<HP> nd;
          load_node(P, p, nd);
          HP dh[6];
#pragma unroll
          for (int c = 0; c < 6; ++c) {
            const HP SL = sc[c], SR = sc[6 + c];
            sp[c] = SL + SR;
            dh[c] = nd.c2 * SL - nd.c1 * SR;
          }
          HP rh[3];
          btvec_hp(nd, dh, rh);  // r_p = B^T (c2 S_L - c1 S_R)
          TF n_[3], c1_, c2_, iwcc, wcc_;
          load_node_tf(P, p, n_, c1_, c2_, iwcc, wcc_);
          const TF rv[3] = {tf_of(rh[0], (TF *)nullptr), tf_of(rh[1], (TF *)nullptr),
                            tf_of(rh[2], (TF *)nullptr)};
          r2 += rv[0] * rv[0] + rv[1] * rv[1] + rv[2] * rv[2];
#pragma unroll
          for (int e = 0; e < 3; ++e) rb_s[3 * t + e] = rv[e] * iwcc;
        }
        __syncthreads();
        const int span = 1 << (K - k);
        const int off = span >> 1;
        const bool owner = (t & (span - 1)) == 0;
        Rec<TF> other;
        if (off >= 32) {
          if ((t & (span - 1)) == off) rec_store(slots + kRecWords * ((t - off) / span), rec);
          __syncthreads();
          if (owner) rec_load(other, slots + kRecWords * (t / span));
          __syncthreads();
        } else {
          rec_shfl_down(other, rec, off, mask, W);
        }
        if (owner) {
          const int p = (1 << K) - (1 << k) + (t >> (K - k));
          TF n[3], c1, c2, iwcc, wcc;
          load_node_tf(P, p, n, c1, c2, iwcc, wcc);
          const int i = t >> (K - k);  // position of node p in its level
          const TF rbv[3] = {rb_s[3 * i], rb_s[3 * i + 1], rb_s[3 * i + 2]};
          combine<TF>(rec, other, n, c1, c2, rbv, gh_s + 21 * p);
        }
      }
      // ---- residual norm, decision (Algorithm 1) ----
      r2 = warp_sum(r2, mask, W);
      const HP ds_ = warp_sum(Dsum, mask, W), xs_ = warp_sum(Xsum, mask, W);
      if (lane == 0) {
        red[warp] = r2;
        redD[warp] = ds_;
        redX[warp] = xs_;
      }
      __syncthreads();
      if (t == 0) {  // in TF: the norm needs no more than a few digits
        TF s = TF(0);
        for (int w = 0; w < nwarp; ++w) s += red[w];
        TF sn = TF(0);
#pragma unroll
        for (int c = 0; c < 6; ++c) {
          const TF v = tf_of(es1[c], (TF *)nullptr);
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
          __syncthreads();
          if (t == 0) {
            ctrl->first = 1;
            ctrl->it = 0;
            ctrl->bt = 0;
            ctrl->gi = TF(1);
            ctrl->res_old = TF(0);
            ctrl->status = 0;
          }
          __syncthreads();
          continue;
        }
        break;
      }
      if (action == ACT_STEP) {
        back_substitute<TF>(P, da_s, gh_s, slots, t);
        __syncthreads();
        for (int i = t; i < 3 * N; i += G) a_s[i] = hp_add_tf(a_s[i], da_s[i]);
      } else {
        const TF f = ctrl->gi * (TF(1) - gamma);
        for (int i = t; i < 3 * N; i += G) a_s[i] = hp_add_tf(a_s[i], -f * da_s[i]);
      }
      __syncthreads();
      if (t == 0 && action == ACT_BACK) {
        ctrl->gi *= gamma;
        ctrl->bt += 1;
      }
    }

    // ---- outputs and state (the last pass is at the final a) ----
    if (t == 0) {
#pragma unroll
      for (int q = 0; q < 21; ++q) orec[q] = rec.C[q];
#pragma unroll
      for (int c = 0; c < 6; ++c) {
        orec[21 + c] = rec.tau[c];
        orec[27 + c] = rec.dd[c];
      }
      orec[33] = rec.gg;
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
    for (int c = t; c < kOutWords; c += G) {  // one output word per thread
      double v;
      if (c < 6) v = hp_to(es1[c]);
      else if (c < 42) v = double(sget(orec, (c - 6) / 6, (c - 6) % 6));
      else if (c < 48) v = double(orec[21 + c - 42]);
      else if (c == 48) v = hp_to(misc[1]);
      else if (c < 55) v = double(orec[27 + c - 49]);
      else if (c == 55) v = double(orec[33]);
      else v = hp_to(misc[2]);
      if (!isfinite(v)) bad = 1;
      P.out[pt * kOutWords + c] = v;
    }
    bad = __syncthreads_or(bad);
    const int bbad = DMN_BOUNDS_CTA_OR();
    if (t == 0) {
      P.status[pt] = (bad ? 2 : ctrl->status) | (attempt ? 4 : 0) | (bbad ? kPtBounds : 0);
      P.iters[pt] = ctrl->it + it_total;
    }
    for (int c = t; c < 8; c += G)  // eps_bar^{n+1} = eps_bar^n + deps exactly in FP64
      sout[c] = c < 6 ? sin[c] + P.deps[pt * 6 + c] : (c == 6 ? theta : 0.0);
    for (int i = t; i < 3 * N; i += G) sout[8 + i] = hp_to(a_s[i]);
    for (int i = t; i < ZW; i += G) sout[8 + 3 * N + i] = hp_to(zw_s[i]);
    for (int i = P.zend + t; i < P.SW; i += G) sout[i] = 0.0;  // padding word
    __syncthreads();
  }
}

static size_t owner_smem_bytes(int K, int zw, int n_mats, bool mixed) {
  const int N = (1 << K) - 1, G = 1 << (K - 1);
  const int nslot = G >= 64 ? G / 64 : 1;
  const size_t hp = 8;  // double or float-float
  size_t b = hp * (3 * N + 9 * G + 2 * zw + 12 + 64 + 4) + sizeof(double) * (nslot * kRecWords);
  b += (mixed ? sizeof(MatPt<float, dfl>) : sizeof(MatPt<double, double>)) * n_mats;
  b = (b + 15) & ~size_t(15);
  b += mixed ? sizeof(Ctrl<float>) : sizeof(Ctrl<double>);
  b += (mixed ? sizeof(float) : sizeof(double)) * (32 + 40 + 24 * N + 3 * (G >= 2 ? G / 2 : 1));
  return (b + 15) & ~size_t(15);
}

// kernel variants: (form, precision, threads bound, CTAs per SM requested).
// 0 = default; 2..4 = owner-mapped mixed kernel for that many CTAs per SM;
// 10 + m = compact kernel (dmn_solve_compact.cu), mixed compiled for m = 2, 3
// or 4 CTAs per SM (11 runs as 12), FP64 for one.  Depth K > 8 takes the
// owner-mapped 512-thread kernel.  A tree with Perzyna leaves (law 2) always
// takes the compact instances that include that leaf law
// (dmn_solve_compact_vp.cu, K <= 9), whatever the variant; one with PA66
// leaves (law 3) the instances of dmn_solve_compact_pa66.cu (K <= 8).
bool is_warp_variant(int variant) { return variant >= 22 && variant <= 24; }
bool solve_variant_valid(int variant) {
  return variant == 0 || (variant >= 2 && variant <= 4) || (variant >= 11 && variant <= 14) ||
         is_warp_variant(variant);
}
static bool uses_warp_form(int K, bool mixed, int variant, int law) {
  return is_warp_variant(variant) && warp_form_supports(K, mixed, law);
}
int solve_block_threads(int K, int variant, int law) {
  (void)law;
  return is_warp_variant(variant) ? 32 * warp_form_warps() : (1 << (K - 1));
}
static bool is_compact(int K, int variant, int law) {
  return law >= 2 ? K <= 9 : (K <= 8 && variant >= 11);
}

static KernelFn pick(int K, bool mixed, int variant, int law) {
  if (uses_warp_form(K, mixed, variant, law)) return warp_kernel(K, variant - 20);
  if (law == 3) return compact_kernel_pa66(K, mixed);
  if (law >= 2) return compact_kernel_vp(K, mixed);
  if (is_compact(K, variant, law)) return compact_kernel(K, mixed, variant - 10);
  if (K > 8) return mixed ? dmn_solve_kernel<float, dfl, 512, 1> : dmn_solve_kernel<double, double, 512, 1>;
  if (!mixed) return dmn_solve_kernel<double, double, 128, 1>;
  switch (variant) {
    case 2: return dmn_solve_kernel<float, dfl, 128, 2>;
    case 4: return dmn_solve_kernel<float, dfl, 128, 4>;
    default: return dmn_solve_kernel<float, dfl, 128, 3>;
  }
}

size_t solve_smem_bytes(int K, int zw, int n_mats, bool mixed, int variant, int law) {
  if (uses_warp_form(K, mixed, variant, law)) return warp_smem_bytes(K, n_mats);
  if (law == 3) return compact_smem_bytes_pa(K, zw, n_mats, mixed);
  return is_compact(K, variant, law) ? compact_smem_bytes(K, zw, n_mats, mixed)
                                     : owner_smem_bytes(K, zw, n_mats, mixed);
}

cudaError_t prepare_solve(int K, int zw, int n_mats, bool mixed, int variant, int law,
                          int *blocks_per_sm) {
  const size_t smem = solve_smem_bytes(K, zw, n_mats, mixed, variant, law);
  KernelFn f = pick(K, mixed, variant, law);
  // One kernel instance serves every tree of a depth range (the compact
  // instances do not depend on K), and its attributes are global to the
  // process: raise them, never lower them, so that a handle prepared for a
  // larger tree (more shared memory, a larger carveout) stays launchable
  // after a smaller tree has been prepared.
  cudaFuncAttributes fa;
  cudaError_t e = cudaFuncGetAttributes(&fa, f);
  if (e != cudaSuccess) return e;
  if (int(smem) > fa.maxDynamicSharedSizeBytes &&
      (e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem))) != cudaSuccess)
    return e;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, f, solve_block_threads(K, variant, law),
                                                          smem)) != cudaSuccess)
    return e;
  // shared memory carveout: the smallest configuration that holds the
  // resident CTAs (plus 1 KB per CTA for the system); the rest of the SM's
  // unified 256 KB stays L1 for the node tables and spills.  The driver
  // rounds a requested percentage up to the next configuration, so request
  // the largest percentage below the chosen one.
  int dev = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
  if (per_sm > 0 && *blocks_per_sm > 0) {
    static const int kConfigKB[] = {0, 8, 16, 32, 64, 100, 132, 164, 196, 228};
    const size_t need = size_t(*blocks_per_sm) * (smem + 1024);
    size_t pick_b = size_t(per_sm);
    for (int kb : kConfigKB)
      if (size_t(kb) * 1024 >= need) {
        pick_b = size_t(kb) * 1024;
        break;
      }
    int pct = pick_b >= size_t(per_sm) ? 100 : int(pick_b * 100 / size_t(per_sm));
    if (pct > fa.preferredShmemCarveout &&
        (e = cudaFuncSetAttribute(f, cudaFuncAttributePreferredSharedMemoryCarveout, pct)) != cudaSuccess)
      return e;
  }
  return cudaSuccess;
}

cudaError_t launch_solve(const SolveParams &P, bool mixed, int variant, int grid, cudaStream_t s) {
  const size_t smem = solve_smem_bytes(P.K, P.zw, P.n_mats, mixed, variant, P.law);
  cudaError_t e = cudaMemsetAsync(P.queue, 0, sizeof(unsigned long long), s);
  if (e != cudaSuccess) return e;
  pick(P.K, mixed, variant, P.law)<<<grid, solve_block_threads(P.K, variant, P.law), smem, s>>>(P);
  return cudaGetLastError();
}

// the index-check log of this translation unit (debug build; dmn_check.cuh)
DMN_BOUNDS_TU(bounds_log_owner)

}  // namespace dmn
