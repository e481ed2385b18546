// dmn_solve.cu -- the Newton solve of Algorithm 1 (arXiv 2109.14403, Sec. 3.3)
// for one Gauss point per CTA.  See dmn_kernels.cuh for the mapping and the
// condensation.
#include "dmn_kernels.cuh"
#include "dmn_internal.h"

namespace dmn {

enum { ACT_STEP = 0, ACT_BACK = 1, ACT_DONE = 2 };

struct Ctrl {
  double res, res_old, gi, r2;
  int action, it, bt, status, first, pad_[3];
};

__device__ __forceinline__ unsigned group_mask(int G) {
  return G >= 32 ? 0xffffffffu : ((1u << G) - 1u);
}
// shuffle segment width: a point with fewer than 32 threads is one segment
__device__ __forceinline__ int group_width(int G) { return G >= 32 ? 32 : G; }

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
        const double *nd = P.node + kNodeWords * p;
        const TF n[3] = {TF(__ldg(nd)), TF(__ldg(nd + 1)), TF(__ldg(nd + 2))};
        const TF c1 = TF(__ldg(nd + 3)), c2 = TF(__ldg(nd + 4));
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

__device__ __forceinline__ double warp_sum(double v, unsigned mask, int W) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1)
    if (o < W) v += __shfl_down_sync(mask, v, o, W);
  return v;
}

// One Newton pass ("Residual" of Algorithm 1 plus the condensation):
//  R1  compact top-down FP64 strain scatter: node j of level k on thread j;
//  R2  thread t: leaves 2t, 2t+1 (FP64 stress, TF record) and laminate t;
//  R3  per level, bottom-up: compact FP64 subtree stress sums and residual
//      r_p = B^T (c2 S_L - c1 S_R), then the owner-mapped TF condensation.
// MAXT bounds the threads per CTA (2^(K-1)); the 128-thread instance (K <= 8)
// lets the compiler use up to 255 registers per thread.
template <typename TF, int MAXT>
__global__ void __launch_bounds__(MAXT) dmn_solve_kernel(const SolveParams P) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int K = P.K, N = P.N, G = P.G;
  const int t = threadIdx.x;
  const int nslot = G >= 64 ? G / 64 : 1;
  double *a_s = reinterpret_cast<double *>(smem_raw);  // 3N  jump vectors
  double *es = a_s + 3 * N;                            // 6N  node strains, then subtree sums
  double *slots = es + 6 * N;                          // nslot * kRecWords
  double *red = slots + nslot * kRecWords;             // 96  warp partial sums
  double *mats_s = red + 96;                           // kMaxMats * 8
  double *eb = mats_s + kMaxMats * 8;                  // 12: eps_bar^{n+1}, deps
  Ctrl *ctrl = reinterpret_cast<Ctrl *>(eb + 12);
  TF *da_s = reinterpret_cast<TF *>(ctrl + 1);         // 3N  Newton increment
  TF *gh_s = da_s + 3 * N;                             // 21N G_p, h_p
  TF *rb_s = gh_s + 21 * N;                            // 3N  residual / (w c1 c2)

  for (int i = t; i < P.n_mats * 8; i += G) mats_s[i] = P.mat[i];
  const unsigned mask = group_mask(G);
  const int W = group_width(G);
  const int lane = t & 31, warp = t >> 5, nwarp = (G + 31) >> 5;

  // per-thread constants: laminate t and its leaves 2t, 2t+1
  const double *nb = P.node + kNodeWords * t;
  const double nbv[3] = {__ldg(nb), __ldg(nb + 1), __ldg(nb + 2)};
  const double c1b = __ldg(nb + 3), c2b = __ldg(nb + 4);
  const TF iwccb = TF(__ldg(nb + 7));
  const double wL = __ldg(P.leafw + 2 * t), wR = __ldg(P.leafw + 2 * t + 1);
  const int j0 = 2 * t, j1 = 2 * t + 1;
  const int zo0 = P.zoff[j0], zo1 = P.zoff[j1];
  const int ph0 = P.phase[j0], ph1 = P.phase[j1];

  for (int64_t pt = blockIdx.x; pt < P.n_points; pt += gridDim.x) {
    const double *sin = P.sin + pt * P.SW;
    double *sout = P.sout + pt * P.SW;
    for (int i = t; i < 3 * N; i += G) a_s[i] = sin[8 + i];
    for (int c = t; c < 6; c += G) {  // a point may have fewer than 6 threads
      const double d = P.deps[pt * 6 + c];
      eb[c] = sin[c] + d;
      eb[6 + c] = d;
    }
    if (t == 0) {
      ctrl->first = 1;
      ctrl->it = 0;
      ctrl->bt = 0;
      ctrl->gi = 1.0;
      ctrl->res_old = 0.0;
      ctrl->status = 0;
    }
    const double theta = P.theta[pt];
    __syncthreads();
    const MatDev &m0 = *reinterpret_cast<const MatDev *>(mats_s + 8 * ph0);
    const MatDev &m1 = *reinterpret_cast<const MatDev *>(mats_s + 8 * ph1);
    const double *zn0 = zo0 >= 0 ? sin + zo0 : nullptr;
    const double *zn1 = zo1 >= 0 ? sin + zo1 : nullptr;

    double trn0 = 0.0, trn1 = 0.0;
    bool first = true;
    double znew0[7] = {0, 0, 0, 0, 0, 0, 0}, znew1[7] = {0, 0, 0, 0, 0, 0, 0};
    double Dsum = 0.0, Xsum = 0.0;
    Rec<TF> rec;
    for (;;) {
      // ---- R1: strains, top-down (eq. DMN kinematics) ----
      for (int c = t; c < 6; c += G) es[6 * (N - 1) + c] = eb[c];
      __syncthreads();
      for (int k = 1; k <= K - 1; ++k) {
        if (t < (1 << (k - 1))) {
          const int p = (1 << K) - (1 << k) + t;
          const int ch = (1 << K) - (1 << (k + 1)) + 2 * t;
          const double *nd = P.node + kNodeWords * p;
          const double n[3] = {__ldg(nd), __ldg(nd + 1), __ldg(nd + 2)};
          const double c1 = __ldg(nd + 3), c2 = __ldg(nd + 4);
          const double av[3] = {a_s[3 * p], a_s[3 * p + 1], a_s[3 * p + 2]};
          double J[6];
          bvec(n, av, J);
#pragma unroll
          for (int c = 0; c < 6; ++c) {
            const double e = es[6 * p + c];
            es[6 * ch + c] = e + c2 * J[c];
            es[6 * ch + 6 + c] = e - c1 * J[c];
          }
        }
        __syncthreads();
      }
      // ---- R2: leaves and laminate t ----
      double r2;
      {
        double e[6], J[6], el[6], er[6];
#pragma unroll
        for (int c = 0; c < 6; ++c) e[c] = es[6 * t + c];
        const double av[3] = {a_s[3 * t], a_s[3 * t + 1], a_s[3 * t + 2]};
        bvec(nbv, av, J);
#pragma unroll
        for (int c = 0; c < 6; ++c) {
          el[c] = e[c] + c2b * J[c];
          er[c] = e[c] - c1b * J[c];
        }
        if (first) {  // at a = a^n: eps^n = eps - deps
          const double trd = eb[6] + eb[7] + eb[8];
          trn0 = (el[0] + el[1] + el[2]) - trd;
          trn1 = (er[0] + er[1] + er[2]) - trd;
        }
        double sl[6], sr[6], DL, DR, XL, XR;
        Rec<TF> rr;
        leaf_eval<TF>(m0, el, theta, zn0, trn0, P.dt, sl, DL, XL, rec, znew0);
        leaf_eval<TF>(m1, er, theta, zn1, trn1, P.dt, sr, DR, XR, rr, znew1);
        Dsum = wL * DL + wR * DR;
        Xsum = wL * XL + wR * XR;
        double d[6], rv[3];
#pragma unroll
        for (int c = 0; c < 6; ++c) {
          const double SL = wL * sl[c], SR = wR * sr[c];
          es[6 * t + c] = SL + SR;
          d[c] = c2b * SL - c1b * SR;
        }
        btvec(nbv, d, rv);
        r2 = rv[0] * rv[0] + rv[1] * rv[1] + rv[2] * rv[2];
        const TF rbv[3] = {TF(rv[0]) * iwccb, TF(rv[1]) * iwccb, TF(rv[2]) * iwccb};
        combine<TF>(rec, rr, nb, rbv, gh_s + 21 * t);
      }
      // ---- R3: bottom-up ----
      for (int k = K - 1; k >= 1; --k) {
        __syncthreads();
        if (t < (1 << (k - 1))) {
          const int p = (1 << K) - (1 << k) + t;
          const int ch = (1 << K) - (1 << (k + 1)) + 2 * t;
          const double *nd = P.node + kNodeWords * p;
          const double n[3] = {__ldg(nd), __ldg(nd + 1), __ldg(nd + 2)};
          const double c1 = __ldg(nd + 3), c2 = __ldg(nd + 4);
          const TF iwcc = TF(__ldg(nd + 7));
          double d[6], rv[3];
#pragma unroll
          for (int c = 0; c < 6; ++c) {
            const double SL = es[6 * ch + c], SR = es[6 * ch + 6 + c];
            es[6 * p + c] = SL + SR;
            d[c] = c2 * SL - c1 * SR;
          }
          btvec(n, d, rv);
          r2 += rv[0] * rv[0] + rv[1] * rv[1] + rv[2] * rv[2];
#pragma unroll
          for (int e = 0; e < 3; ++e) rb_s[3 * p + e] = TF(rv[e]) * iwcc;
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
          const TF rbv[3] = {rb_s[3 * p], rb_s[3 * p + 1], rb_s[3 * p + 2]};
          combine<TF>(rec, other, P.node + kNodeWords * p, rbv, gh_s + 21 * p);
        }
      }
      // ---- residual norm, decision (Algorithm 1) ----
      r2 = warp_sum(r2, mask, W);
      const double ds_ = warp_sum(Dsum, mask, W), xs_ = warp_sum(Xsum, mask, W);
      if (lane == 0) {
        red[warp] = r2;
        red[32 + warp] = ds_;
        red[64 + warp] = xs_;
      }
      __syncthreads();
      if (t == 0) {
        double s = 0.0;
        for (int w = 0; w < nwarp; ++w) s += red[w];
        double sn = 0.0;
#pragma unroll
        for (int c = 0; c < 6; ++c) sn += es[6 * (N - 1) + c] * es[6 * (N - 1) + c];
        double den = sqrt(sn);
        if (den < P.res_floor) den = P.res_floor;
        const double res = sqrt(s) / (double(N) * den);
        Ctrl &c = *ctrl;
        const bool accept = c.first || (res < c.res_old) || (c.bt >= P.maxbt);
        int action;
        if (accept) {
          if (!isfinite(res)) {
            c.status = 2;
            action = ACT_DONE;
          } else if (!c.first && res < P.tol) {
            c.status = 0;
            action = ACT_DONE;
          } else if (c.it >= P.maxit) {
            c.status = 1;
            action = ACT_DONE;
          } else {
            c.res_old = res;
            c.it += 1;
            c.bt = 0;
            c.gi = 1.0;
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
      if (action == ACT_DONE) break;
      if (action == ACT_STEP) {
        back_substitute<TF>(P, da_s, gh_s, slots, t);
        __syncthreads();
        for (int i = t; i < 3 * N; i += G) a_s[i] += double(da_s[i]);
      } else {
        const double f = ctrl->gi * (1.0 - P.gamma);
        for (int i = t; i < 3 * N; i += G) a_s[i] -= f * double(da_s[i]);
      }
      __syncthreads();
      if (t == 0 && action == ACT_BACK) {
        ctrl->gi *= P.gamma;
        ctrl->bt += 1;
      }
    }

    // ---- outputs and state (the last pass is at the final a) ----
    if (t == 0) {
      double *o = P.out + pt * kOutWords;
      int st = ctrl->status;
      double v[kOutWords];
#pragma unroll
      for (int c = 0; c < 6; ++c) v[c] = es[6 * (N - 1) + c];
#pragma unroll
      for (int i = 0; i < 6; ++i)
#pragma unroll
        for (int j = 0; j < 6; ++j) v[6 + 6 * i + j] = double(sget(rec.C, i, j));
#pragma unroll
      for (int c = 0; c < 6; ++c) v[42 + c] = double(rec.tau[c]);
      double Db = 0.0, Xb = 0.0;
      for (int w = 0; w < nwarp; ++w) {
        Db += red[32 + w];
        Xb += red[64 + w];
      }
      v[48] = Db;
#pragma unroll
      for (int c = 0; c < 6; ++c) v[49 + c] = double(rec.dd[c]);
      v[55] = double(rec.gg);
      v[56] = Xb;
      for (int c = 0; c < kOutWords; ++c) {
        if (!isfinite(v[c])) st = 2;
        o[c] = v[c];
      }
      P.status[pt] = st;
      P.iters[pt] = ctrl->it;
    }
    for (int c = t; c < 8; c += G) sout[c] = c < 6 ? eb[c] : (c == 6 ? theta : 0.0);
    for (int i = t; i < 3 * N; i += G) sout[8 + i] = a_s[i];
    if (zo0 >= 0) {
#pragma unroll
      for (int c = 0; c < 7; ++c) sout[zo0 + c] = znew0[c];
    }
    if (zo1 >= 0) {
#pragma unroll
      for (int c = 0; c < 7; ++c) sout[zo1 + c] = znew1[c];
    }
    for (int i = P.zend + t; i < P.SW; i += G) sout[i] = 0.0;  // padding word
    __syncthreads();
  }
}

size_t solve_smem_bytes(int K, bool mixed) {
  const int N = (1 << K) - 1, G = 1 << (K - 1);
  const int nslot = G >= 64 ? G / 64 : 1;
  size_t b = sizeof(double) * (9 * N + nslot * kRecWords + 96 + kMaxMats * 8 + 12) + sizeof(Ctrl);
  b += (mixed ? sizeof(float) : sizeof(double)) * (27 * N);
  return (b + 15) & ~size_t(15);
}

template <typename TF, int MAXT>
static cudaError_t prepare_t(int K, int *blocks_per_sm) {
  const size_t smem = solve_smem_bytes(K, sizeof(TF) == 4);
  cudaError_t e = cudaFuncSetAttribute(dmn_solve_kernel<TF, MAXT>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, dmn_solve_kernel<TF, MAXT>,
                                                       1 << (K - 1), smem);
}

cudaError_t prepare_solve(int K, bool mixed, int *blocks_per_sm) {
  if (K <= 8)
    return mixed ? prepare_t<float, 128>(K, blocks_per_sm) : prepare_t<double, 128>(K, blocks_per_sm);
  return mixed ? prepare_t<float, 512>(K, blocks_per_sm) : prepare_t<double, 512>(K, blocks_per_sm);
}

cudaError_t launch_solve(const SolveParams &P, bool mixed, int grid, cudaStream_t s) {
  const size_t smem = solve_smem_bytes(P.K, mixed);
  if (P.K <= 8) {
    if (mixed) dmn_solve_kernel<float, 128><<<grid, P.G, smem, s>>>(P);
    else dmn_solve_kernel<double, 128><<<grid, P.G, smem, s>>>(P);
  } else {
    if (mixed) dmn_solve_kernel<float, 512><<<grid, P.G, smem, s>>>(P);
    else dmn_solve_kernel<double, 512><<<grid, P.G, smem, s>>>(P);
  }
  return cudaGetLastError();
}

}  // namespace dmn
