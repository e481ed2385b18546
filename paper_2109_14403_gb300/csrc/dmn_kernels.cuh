// dmn_kernels.cuh -- device code of the DMN online evaluation (arXiv 2109.14403,
// Sec. 3.3, Algorithm 1) for sm_103a.
//
// Mapping: one CTA per Gauss point (grid-stride over points), G = 2^(K-1)
// threads; thread t owns the bottom laminate t (paper index t) and its two
// leaves 2t, 2t+1.  A node (level k, position i) is owned by thread
// i * 2^(K-k), the owner of its leftmost bottom laminate.
//
// Newton system (eq. Newton) by exact hierarchical condensation.  For a fixed
// strain perturbation e of a node, the minimum of the quadratic Newton model of
// its subtree is 1/2 e.C_hat e + s_hat.e, with
//   K_p   = B^T (c2 C_L + c1 C_R) B                     (3x3, SPD)
//   a_p   = -K_p^{-1} B^T (dC e + ds),   dC = C_L - C_R, ds = s_L - s_R
//   C_hat = c1 C_L + c2 C_R - c1 c2 dC B K_p^{-1} B^T dC
//   s_hat = c1 s_L + c2 s_R - c1 c2 dC B K_p^{-1} B^T ds
// where B a = sym(a (x) n_p).  This is the block elimination of
// A^T W dsigma/deps A in postorder; with e = 0 at the root a top-down sweep
// gives the Newton increment exactly.  The same recursion applied to
// dsigma/dtheta, dD/deps and dD/dtheta gives the four algorithmic tangents at
// the root (eqs. ddsdde, ddsddt, drplde, drpldt) without extra right-hand
// sides.  The residual A^T W sigma of Algorithm 1 is, node by node,
//   r_p = w_p c1 c2 B^T (sigma_bar_L - sigma_bar_R)
// with sigma_bar the plain weighted mean stress of a subtree (FP64).
//
// Precision: TF = double (every step FP64) or float (mixed).  In mixed mode
// the condensed stress is carried as sigma_bar (FP64) + a TF correction, so
// the Newton right-hand side is formed from FP64 stress differences and only
// the O(residual) correction is rounded to FP32.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "dfl.cuh"
#include "dmn_check.cuh"

namespace dmn {

constexpr double kRsq2 = 0.70710678118654752440;
constexpr int kMaxMats = 16;
constexpr int kOutWords = 57;
constexpr int kNodeWords = 12;  // FP64 node table row
constexpr int kNodeDfl = 20;    // float-float node table row (floats)

constexpr int kPaBranches = 12;  // Maxwell branches of the PA66 leaf
constexpr int kPaZ = 7 + 6 * kPaBranches;  // its internal variables in the state
constexpr int kPaHist = 34;  // its history words in the solve's shared memory
constexpr int kMatWords = 40;  // device material row
// Kinds 0-2 use the first 12 words.  Kind 3 (PA66): Kb, G of the long-term
// branch, alpha, theta0, sy0, then dsy = k (hardening), H = n (exponent),
// mexp = m, itv = eta0, cE = beta1, pad_ = beta2, and pa = theta_ref, C1, C2,
// nu, E_1..E_12, tau_1..tau_12.
struct MatDev {
  double kind, Kb, G, alpha, theta0, sy0, dsy, H;  // moduli at theta0
  double mexp, itv, cE, pad_;  // Perzyna: rate exponent, 1 / t_visc, dE_dT / E
  double pa[28];
};

struct SolveParams {
  int K, N, G, SW;         // depth, nodes, threads per point, state words
  int n_mats, maxit, maxbt, zend;  // zend: end of the z data in a state block
  int zw;                          // words of internal variables per state block
  int law;                         // largest material kind of the tree (1, 2 or 3)
  const int *hoff;                 // law 3: offset of a leaf's history in shared memory, -1 none
  unsigned long long *queue;       // device counter of points taken (zeroed per launch)
  const float *da0;                // optional warm-start increment [n][3N] (NULL: start at a^n)
  const int *skip;                 // optional [n]: points with skip[i] != 0 are left untouched
  double tol, gamma, res_floor, dt;
  const double *node;      // [N][kNodeWords]: n0 n1 n2 c1 c2 w w*c1*c2 1/(w*c1*c2)
                           //   n0/sqrt2 n1/sqrt2 n2/sqrt2 0
  const float *node_df;    // [N][kNodeDfl]: (hi, lo) of n0 n1 n2 n0/sqrt2 n1/sqrt2
                           //   n2/sqrt2 c1 c2, then 1/(w c1 c2) and padding
  const double *leafw;     // [2^K] leaf weights
  const uint8_t *phase;    // [2^K]
  const int *zoff;         // [2^K]: offset of the leaf's z in a state block, -1 none
  const double *mat;       // [n_mats][kMatWords] as MatDev
  int64_t n_points;
  const double *deps, *theta, *sin;
  double *sout, *out;
  int *status, *iters;
  float *gh;               // warp form: per-warp slots of the lanes' G_p, h_p (scratch)
};

// ------------------------------------------------------------------ helpers
__host__ __device__ constexpr int sidx(int i, int j) {
  // packed upper triangle of a symmetric 6x6, i <= j
  return i * 6 - (i * (i - 1)) / 2 + (j - i);
}
template <typename T>
__device__ __forceinline__ T sget(const T *S, int i, int j) {
  return i <= j ? S[sidx(i, j)] : S[sidx(j, i)];
}

// B a = sym(a (x) n) as a Mandel vector
template <typename T>
__device__ __forceinline__ void bvec(const T n[3], const T a[3], T out[6]) {
  const T r = T(kRsq2);
  out[0] = a[0] * n[0];
  out[1] = a[1] * n[1];
  out[2] = a[2] * n[2];
  out[3] = r * (a[1] * n[2] + a[2] * n[1]);
  out[4] = r * (a[0] * n[2] + a[2] * n[0]);
  out[5] = r * (a[0] * n[1] + a[1] * n[0]);
}
// B^T s = s n (traction)
template <typename T>
__device__ __forceinline__ void btvec(const T n[3], const T s[6], T out[3]) {
  const T r = T(kRsq2);
  out[0] = s[0] * n[0] + r * (s[5] * n[1] + s[4] * n[2]);
  out[1] = s[1] * n[1] + r * (s[5] * n[0] + s[3] * n[2]);
  out[2] = s[2] * n[2] + r * (s[4] * n[0] + s[3] * n[1]);
}

// condensed record of a subtree (or a leaf), condensation precision TF
template <typename TF>
struct Rec {
  TF C[21];       // condensed tangent
  TF ds[6];       // condensed stress minus the plain weighted mean stress
  TF tau[6];      // condensed d sigma / d theta
  TF dd[6];       // condensed d D / d eps
  TF gg;          // condensed d D / d theta
};
constexpr int kRecWords = 40;  // exchange slot in doubles

// ------------------------------------------------------------------ phase laws
// Constants of one material.  The static part is built once per CTA (FP64 is
// fine there); the part that depends on the point's temperature theta is
// formed per point in the high-precision type HP, so the mixed path stays on
// the FP32 pipe.  Kind 2 (Perzyna) scales its moduli with theta per point.
template <typename TF, typename HP>
struct MatPt {
  HP Kb, G2, G3, iden, H, a3K, alpha, theta0, sy0, dsy, symin, third, c15, one;
  TF a3K_f, G2_f, G3_f, Kb_f, iden_f, dsy0_f;
  int kind, mexp;
  // kind 2, static: moduli at theta0, modulus slope, c = dt / t_visc, floor of r
  HP Kb0, G20, G30, a3K0, cE, cvisc, rmin;
  TF cvisc_f, cE_f, Kb0_f, H_f;
  // per point
  HP ath;        // alpha (theta - theta0)
  HP a3Kth_idt;  // 3 K alpha theta / dt
  HP sy, syidt;  // sigma_Y(theta) (floored at 1e-6 MPa), sigma_Y / dt
  TF a3K_idt_f, dsy_f, sy_f, idt_f;
  // per point, kind 2
  HP isy, thsE_idt;  // 1 / sigma_Y, theta (r'/r) / dt
  TF sE_f, th_f, dKb_f, thsE_idt_f, gj_f, af_f;  // r'/r, theta, dK/dtheta, ..., 3 alpha dK/dtheta theta / dt, 3G + H
};

template <typename TF, typename HP>
__device__ __forceinline__ void mat_static(MatPt<TF, HP> &o, const MatDev &m, double dt) {
  HP *tag = nullptr;
  const double den = 3.0 * m.G + m.H;
  o.Kb = hp_from(m.Kb, tag);
  o.G2 = hp_from(2.0 * m.G, tag);
  o.G3 = hp_from(3.0 * m.G, tag);
  o.iden = hp_from(1.0 / den, tag);
  o.H = hp_from(m.H, tag);
  o.a3K = hp_from(3.0 * m.Kb * m.alpha, tag);
  o.alpha = hp_from(m.alpha, tag);
  o.theta0 = hp_from(m.theta0, tag);
  o.sy0 = hp_from(m.sy0, tag);
  o.dsy = hp_from(m.dsy, tag);
  o.symin = hp_from(1e-6, tag);
  o.third = hp_from(1.0 / 3.0, tag);
  o.c15 = hp_from(1.5, tag);
  o.one = hp_from(1.0, tag);
  o.a3K_f = TF(3.0 * m.Kb * m.alpha);
  o.G2_f = TF(2.0 * m.G);
  o.G3_f = TF(3.0 * m.G);
  o.Kb_f = TF(m.Kb);
  o.iden_f = TF(1.0 / den);
  o.dsy0_f = TF(m.dsy);
  o.kind = int(m.kind + 0.5);
  o.mexp = int(m.mexp + 0.5);
  o.Kb0 = o.Kb;
  o.G20 = o.G2;
  o.G30 = o.G3;
  o.a3K0 = o.a3K;
  o.cE = hp_from(m.cE, tag);
  o.cvisc = hp_from(dt * m.itv, tag);
  o.rmin = hp_from(1e-3, tag);
  o.cvisc_f = TF(dt * m.itv);
  o.cE_f = TF(m.cE);
  o.Kb0_f = TF(m.Kb);
  o.H_f = TF(m.H);
}

template <typename TF, typename HP, int LAW>
__device__ __forceinline__ void mat_point(MatPt<TF, HP> &o, HP theta, HP idt, TF idt_f) {
  const HP dth = theta - o.theta0;
  if (LAW >= 2 && o.kind == 2) {
    // moduli E (1 + dE_dT (theta - theta0)), the factor floored at 1e-3
    HP r = o.one + o.cE * dth;
    TF dr = o.cE_f;
    if (tf_of(r, (TF *)nullptr) < TF(1e-3)) {
      r = o.rmin;
      dr = TF(0);
    }
    o.Kb = o.Kb0 * r;
    o.G2 = o.G20 * r;
    o.G3 = o.G30 * r;
    o.a3K = o.a3K0 * r;
    o.Kb_f = tf_of(o.Kb, (TF *)nullptr);
    o.G2_f = tf_of(o.G2, (TF *)nullptr);
    o.G3_f = tf_of(o.G3, (TF *)nullptr);
    o.a3K_f = tf_of(o.a3K, (TF *)nullptr);
    o.af_f = o.G3_f + o.H_f;
    o.iden_f = TF(1) / o.af_f;
    const TF rf = tf_of(r, (TF *)nullptr);
    o.sE_f = dr / rf;
    o.th_f = tf_of(theta, (TF *)nullptr);
    o.dKb_f = o.Kb0_f * dr;
    o.thsE_idt_f = o.th_f * o.sE_f * idt_f;
    o.gj_f = TF(3) * tf_of(o.alpha, (TF *)nullptr) * o.dKb_f * o.th_f * idt_f;
    o.thsE_idt = dr == TF(0) ? hp_zero((HP *)nullptr) : hp_div(o.cE * theta * idt, r);
  }
  o.ath = o.alpha * dth;
  o.a3Kth_idt = o.a3K * theta * idt;
  HP sy = o.sy0 + o.dsy * dth;
  TF dsy = o.dsy0_f;
  if (tf_of(sy, (TF *)nullptr) < TF(1e-6)) {
    sy = o.symin;
    dsy = TF(0);
  }
  o.sy = sy;
  o.syidt = sy * idt;
  o.a3K_idt_f = o.a3K_f * idt_f;
  o.dsy_f = dsy;
  o.sy_f = tf_of(sy, (TF *)nullptr);
  o.idt_f = idt_f;
  if (LAW >= 2 && o.kind == 2) o.isy = hp_div(o.one, sy);
}

// Leaf update at strain eps and the point's temperature (Sec. 4).  Stress,
// coupling term D and dissipation X in HP; derivatives into the TF record.
// zn = internal variables at t^n (eps_p Mandel 6, p; kind 2 also the leaf
// strain at t^n), trn = trace of the leaf strain at t^n (kinds 0 and 1).
// J2 radial return with linear hardening, written as
// sigma = K tr(ee) I + th1 s_tr, d eps_p = (3/2)(dp/q_tr) s_tr, th1 = 1 - 3G dp/q_tr;
// the yield test compares squares, so elastic leaves take no square root.
// Kind 2 (LAW >= 2): dp solves the implicit Euler step of the overstress law,
// dp = c phi^m, phi = (q_tr - (3G + H) dp - sigma_Y - H p^n) / sigma_Y, by
// Newton in TF (g concave and increasing: monotone from dp = 0) and two
// Newton corrections in HP; the tangent is the radial-return one with
// 1/(3G + H) replaced by c m phi^(m-1) / (sigma_Y + c m phi^(m-1) (3G + H));
// temperature-dependent moduli add theta (r'/r) sigma : (de - d eps_p) / dt
// to D, de the leaf's strain increment.  With full = false the output-only
// quantities (D, X and the record's tau, dd, gg) are left at zero.
template <typename TF, typename HP, int LAW>
__device__ __forceinline__ void leaf_eval(const MatPt<TF, HP> &m, const HP eps[6], const HP *zn,
                                          HP trn, HP sig[6], HP &D, HP &X, Rec<TF> &R, HP *znew,
                                          bool full = true) {
  const bool j2 = m.kind >= 1;
  const bool vp = LAW >= 2 && m.kind == 2;
  HP ee[6];
#pragma unroll
  for (int c = 0; c < 6; ++c) {
    ee[c] = c < 3 ? eps[c] - m.ath : eps[c];
    if (j2) ee[c] = ee[c] - zn[c];
  }
  const HP tr = ee[0] + ee[1] + ee[2];
  const HP tr3 = tr * m.third;
  HP s[6];
#pragma unroll
  for (int c = 0; c < 6; ++c) s[c] = m.G2 * (c < 3 ? ee[c] - tr3 : ee[c]);
  const HP pk = m.Kb * tr;
  HP dtr = hp_zero((HP *)nullptr);
  HP de[6];
  D = hp_zero((HP *)nullptr);
  X = hp_zero((HP *)nullptr);
  TF gg = TF(0);
  if (full) {
    if (vp) {
#pragma unroll
      for (int c = 0; c < 6; ++c) de[c] = eps[c] - zn[7 + c];
      dtr = de[0] + de[1] + de[2];
    } else {
      const HP treps = eps[0] + eps[1] + eps[2];
      dtr = treps - trn;
    }
    D = -(m.a3Kth_idt * dtr);
    gg = -m.a3K_idt_f * tf_of(dtr, (TF *)nullptr);
    if (vp) gg -= m.gj_f * tf_of(dtr, (TF *)nullptr);
  }
  TF th1 = TF(1), thb = TF(0), kd = TF(0), ktau = TF(0);
  TF Nf[6] = {TF(0), TF(0), TF(0), TF(0), TF(0), TF(0)};
  TF qf = TF(0), kkf = TF(0), ddpf = TF(0);  // kind 2: q, d dp / d eps factor, d dp / d theta
  HP kzs = hp_zero((HP *)nullptr);           // kind 2: d eps_p = kzs s_tr
  bool plastic = false;
  if (j2) {
    HP sn2 = s[0] * s[0];
#pragma unroll
    for (int c = 1; c < 6; ++c) sn2 = sn2 + s[c] * s[c];
    const HP yr = m.sy + m.H * zn[6];
    const HP q2 = m.c15 * sn2;
    plastic = hp_gt(q2, yr * yr);
    if (plastic) {
      const HP q = hp_sqrt(q2);  // q_tr = sqrt(3/2) |s_tr|
      HP dp;
      TF kinv = m.iden_f, phif = TF(0);
      if (vp) {
        const HP f = q - yr;
        const TF ff = tf_of(f, (TF *)nullptr), af = m.af_f, isyf = TF(1) / m.sy_f;
        const TF cf = m.cvisc_f, xmax = ff / af;
        const int me = m.mexp;
        TF x = TF(0), gp = TF(1);
        for (int it = 0; it < 64; ++it) {
          TF phi = (ff - af * x) * isyf;
          if (phi < TF(0)) phi = TF(0);
          TF pw = TF(1);
          for (int k = 1; k < me; ++k) pw *= phi;  // phi^(m-1)
          const TF gx = x - cf * pw * phi;
          gp = TF(1) + cf * TF(me) * pw * af * isyf;
          TF xn = x - gx / gp;
          if (xn < TF(0)) xn = TF(0);
          if (xn > xmax) xn = xmax;
          const TF step = fabs(xn - x);
          x = xn;
          if (!(step > TF(sizeof(TF) == 4 ? 1e-7 : 1e-15) * x)) break;
        }
        // two corrections in HP with the TF derivative
        dp = hp_add_tf(hp_zero((HP *)nullptr), x);
        const TF igp = TF(1) / gp;
        for (int k2 = 0; k2 < 2; ++k2) {
          HP ph = (f - (m.G3 + m.H) * dp) * m.isy;
          if (tf_of(ph, (TF *)nullptr) < TF(0)) ph = hp_zero((HP *)nullptr);
          HP pwm = ph;
          for (int k = 1; k < me; ++k) pwm = pwm * ph;  // phi^m
          const HP g = dp - m.cvisc * pwm;
          dp = dp - g * igp;
        }
        phif = tf_of((f - (m.G3 + m.H) * dp) * m.isy, (TF *)nullptr);
        if (phif < TF(0)) phif = TF(0);
        TF pw = TF(1);
        for (int k = 1; k < me; ++k) pw *= phif;
        const TF cm = cf * TF(me) * pw;
        kinv = cm / (m.sy_f + cm * af);  // 1 / (3G + H + h_v)
      } else {
        dp = (q - yr) * m.iden;  // closed-form plastic multiplier
      }
      const HP kap = hp_div(dp, q);  // dp / q_tr
      const HP th1h = m.one - m.G3 * kap;
      const HP kz = m.c15 * kap;
#pragma unroll
      for (int c = 0; c < 6; ++c) {
        sig[c] = c < 3 ? pk + th1h * s[c] : th1h * s[c];
        znew[c] = zn[c] + kz * s[c];
      }
      znew[6] = zn[6] + dp;
      kzs = kz;
      if (full) {
        const HP dis = m.syidt * dp;
        D = D + dis;
        X = dis;
      }
      const TF kapf = tf_of(kap, (TF *)nullptr), dpf = tf_of(dp, (TF *)nullptr);
      th1 = TF(1) - m.G3_f * kapf;
      thb = m.G3_f * kinv - m.G3_f * kapf;
      const TF isn = TF(1) / sqrt(tf_of(sn2, (TF *)nullptr));
#pragma unroll
      for (int c = 0; c < 6; ++c) Nf[c] = tf_of(s[c], (TF *)nullptr) * isn;
      if (!full) {
      } else if (vp) {
        qf = tf_of(q, (TF *)nullptr) - m.G3_f * dpf;  // updated equivalent stress
        ddpf = (m.sE_f * qf - m.dsy_f * (TF(1) + phif)) * kinv;
        ktau = TF(0.81649658092772603273) * (m.sE_f * qf - m.G3_f * ddpf);  // sqrt(2/3) dq/dtheta
        kkf = TF(1.2247448713915890491) * m.G2_f * kinv;
        kd = m.sy_f * kkf * m.idt_f;
        gg += (m.dsy_f * dpf + m.sy_f * ddpf) * m.idt_f;
      } else {
        ktau = m.G2_f * TF(1.2247448713915890491) * m.dsy_f * m.iden_f;
        kd = m.sy_f * TF(1.2247448713915890491) * m.G2_f * m.iden_f * m.idt_f;
        gg += (m.dsy_f * dpf - m.sy_f * m.dsy_f * m.iden_f) * m.idt_f;
      }
    } else {
#pragma unroll
      for (int c = 0; c < 7; ++c) znew[c] = zn[c];
    }
    if (vp) {
#pragma unroll
      for (int c = 0; c < 6; ++c) znew[7 + c] = eps[c];
    }
  }
  if (!plastic) {
#pragma unroll
    for (int c = 0; c < 6; ++c) sig[c] = c < 3 ? pk + s[c] : s[c];
  }
  // tangent C = 3K P1 + 2G th1 P2 - 2G thb N (x) N
  const TF cP1 = m.Kb_f - m.G2_f * th1 / TF(3);  // coefficient of m m^T
  const TF cI = m.G2_f * th1;
  const TF cN = m.G2_f * thb;
#pragma unroll
  for (int i = 0; i < 6; ++i)
#pragma unroll
    for (int j = i; j < 6; ++j)
      R.C[sidx(i, j)] = (i < 3 && j < 3 ? cP1 : TF(0)) + (i == j ? cI : TF(0)) - cN * Nf[i] * Nf[j];
#pragma unroll
  for (int c = 0; c < 6; ++c) {
    R.ds[c] = TF(0);
    R.tau[c] = TF(0);
    R.dd[c] = TF(0);
  }
  R.gg = TF(0);
  if (!full) return;
  TF ta = -m.a3K_f;
  if (vp) ta += m.dKb_f * tf_of(tr, (TF *)nullptr);
  const TF da_ = -tf_of(m.a3Kth_idt, (TF *)nullptr);
#pragma unroll
  for (int c = 0; c < 6; ++c) {
    R.tau[c] = (c < 3 ? ta : TF(0)) + ktau * Nf[c];
    R.dd[c] = (c < 3 ? da_ : TF(0)) + kd * Nf[c];
  }
  if (vp) {
    // elastic leaf: the deviatoric stress scales with the moduli
    if (!plastic) {
#pragma unroll
      for (int c = 0; c < 6; ++c) R.tau[c] += m.sE_f * tf_of(s[c], (TF *)nullptr);
    }
    // theta (r'/r) sigma : v / dt with v = de - d eps_p, and its derivatives
    HP v[6];
#pragma unroll
    for (int c = 0; c < 6; ++c) v[c] = plastic ? de[c] - kzs * s[c] : de[c];
    HP sv = sig[0] * v[0];
#pragma unroll
    for (int c = 1; c < 6; ++c) sv = sv + sig[c] * v[c];
    D = D + m.thsE_idt * sv;
    TF vf[6];
#pragma unroll
    for (int c = 0; c < 6; ++c) vf[c] = tf_of(v[c], (TF *)nullptr);
    const TF mv = vf[0] + vf[1] + vf[2];
    TF Nv = TF(0), tv = TF(0);
#pragma unroll
    for (int c = 0; c < 6; ++c) {
      Nv += Nf[c] * vf[c];
      tv += R.tau[c] * vf[c];
    }
#pragma unroll
    for (int c = 0; c < 6; ++c) {
      const TF Cv = (c < 3 ? cP1 * mv : TF(0)) + cI * vf[c] - cN * Nf[c] * Nv;
      R.dd[c] += m.thsE_idt_f * (Cv + tf_of(sig[c], (TF *)nullptr) - qf * kkf * Nf[c]);
    }
    const TF svf = tf_of(sv, (TF *)nullptr);
    gg += m.sE_f * (TF(1) - m.th_f * m.sE_f) * svf * m.idt_f + m.thsE_idt_f * (tv - qf * ddpf);
  }
  R.gg = gg;
}

// ------------------------------------------------------------------ condensation
// Combine children L (in/out) and R of node p in precision TF.  rbv =
// B^T (sigma_bar_L - sigma_bar_R), the node's residual divided by w c1 c2
// (formed in FP64 by the caller).  Writes G_p (3x6) and h_p (3) for the
// back-substitution.  With full = false the output-only parts of the record
// (tau, dd, gg) are not formed.
template <typename TF>
__device__ __forceinline__ void combine(Rec<TF> &L, const Rec<TF> &R, const TF n[3], TF c1, TF c2,
                                        const TF rbv[3], TF *gh, bool full = true) {
  const TF cc = c1 * c2;
  // M = c2 C_L + c1 C_R, dC = C_L - C_R (dC in place of L.C)
  TF M[21];
#pragma unroll
  for (int q = 0; q < 21; ++q) {
    M[q] = c2 * L.C[q] + c1 * R.C[q];
    L.C[q] = L.C[q] - R.C[q];
  }
  // K = B^T M B
  TF MB[6][3];
#pragma unroll
  for (int a = 0; a < 6; ++a) {
    TF row[6];
#pragma unroll
    for (int b = 0; b < 6; ++b) row[b] = sget(M, a, b);
    btvec(n, row, MB[a]);
  }
  TF Kk[3][3];
#pragma unroll
  for (int f = 0; f < 3; ++f) {
    TF col[6], t3[3];
#pragma unroll
    for (int a = 0; a < 6; ++a) col[a] = MB[a][f];
    btvec(n, col, t3);
#pragma unroll
    for (int e = 0; e < 3; ++e) Kk[e][f] = t3[e];
  }
  // K^{-1} by the adjugate (K is SPD 3x3)
  const TF k00 = Kk[0][0], k11 = Kk[1][1], k22 = Kk[2][2];
  const TF k01 = TF(0.5) * (Kk[0][1] + Kk[1][0]);
  const TF k02 = TF(0.5) * (Kk[0][2] + Kk[2][0]);
  const TF k12 = TF(0.5) * (Kk[1][2] + Kk[2][1]);
  const TF a00 = k11 * k22 - k12 * k12, a01 = k02 * k12 - k01 * k22, a02 = k01 * k12 - k02 * k11;
  const TF a11 = k00 * k22 - k02 * k02, a12 = k01 * k02 - k00 * k12, a22 = k00 * k11 - k01 * k01;
  const TF idet = TF(1) / (k00 * a00 + k01 * a01 + k02 * a02);
  const TF Ki[3][3] = {{a00 * idet, a01 * idet, a02 * idet},
                       {a01 * idet, a11 * idet, a12 * idet},
                       {a02 * idet, a12 * idet, a22 * idet}};
  // U = dC B (6x3), G = K^{-1} U^T (3x6)
  TF U[6][3];
#pragma unroll
  for (int a = 0; a < 6; ++a) {
    TF row[6];
#pragma unroll
    for (int b = 0; b < 6; ++b) row[b] = sget(L.C, a, b);
    btvec(n, row, U[a]);
  }
  TF Gm[3][6];
#pragma unroll
  for (int e = 0; e < 3; ++e)
#pragma unroll
    for (int a = 0; a < 6; ++a) Gm[e][a] = Ki[e][0] * U[a][0] + Ki[e][1] * U[a][1] + Ki[e][2] * U[a][2];
  // condensed stress: B^T ds_hat = rb + B^T (ds_L - ds_R)
  TF hs[3];
  {
    TF dds[6], t3[3];
#pragma unroll
    for (int c = 0; c < 6; ++c) dds[c] = L.ds[c] - R.ds[c];
    btvec(n, dds, t3);
    TF b3[3];
#pragma unroll
    for (int e = 0; e < 3; ++e) b3[e] = rbv[e] + t3[e];
#pragma unroll
    for (int e = 0; e < 3; ++e) hs[e] = Ki[e][0] * b3[0] + Ki[e][1] * b3[1] + Ki[e][2] * b3[2];
  }
#pragma unroll
  for (int e = 0; e < 3; ++e)
#pragma unroll
    for (int a = 0; a < 6; ++a) gh[6 * e + a] = Gm[e][a];
#pragma unroll
  for (int e = 0; e < 3; ++e) gh[18 + e] = hs[e];
#pragma unroll
  for (int a = 0; a < 6; ++a) {
    const TF Uhs = U[a][0] * hs[0] + U[a][1] * hs[1] + U[a][2] * hs[2];
    L.ds[a] = c1 * L.ds[a] + c2 * R.ds[a] - cc * Uhs;
  }
  if (full) {
    TF ht[3];
    {
      TF dv[6], t3[3];
#pragma unroll
      for (int c = 0; c < 6; ++c) dv[c] = L.tau[c] - R.tau[c];
      btvec(n, dv, t3);
#pragma unroll
      for (int e = 0; e < 3; ++e) ht[e] = Ki[e][0] * t3[0] + Ki[e][1] * t3[1] + Ki[e][2] * t3[2];
    }
    TF hd[3], bd[3];
    {
      TF ddiff[6];
#pragma unroll
      for (int c = 0; c < 6; ++c) ddiff[c] = L.dd[c] - R.dd[c];
      btvec(n, ddiff, bd);
#pragma unroll
      for (int e = 0; e < 3; ++e) hd[e] = Ki[e][0] * bd[0] + Ki[e][1] * bd[1] + Ki[e][2] * bd[2];
    }
    // g_hat = c1 g_L + c2 g_R - c1 c2 (B^T d_diff) . h_tau
    L.gg = c1 * L.gg + c2 * R.gg - cc * (bd[0] * ht[0] + bd[1] * ht[1] + bd[2] * ht[2]);
#pragma unroll
    for (int a = 0; a < 6; ++a) {
      const TF Uht = U[a][0] * ht[0] + U[a][1] * ht[1] + U[a][2] * ht[2];
      const TF Uhd = U[a][0] * hd[0] + U[a][1] * hd[1] + U[a][2] * hd[2];
      L.tau[a] = c1 * L.tau[a] + c2 * R.tau[a] - cc * Uht;
      L.dd[a] = c1 * L.dd[a] + c2 * R.dd[a] - cc * Uhd;
    }
  }
  // C_hat = c1 C_L + c2 C_R - c1 c2 U G  with c1 C_L + c2 C_R = M + (c1 - c2) dC
  const TF cm = c1 - c2;
#pragma unroll
  for (int i = 0; i < 6; ++i)
#pragma unroll
    for (int j = i; j < 6; ++j) {
      const int q = sidx(i, j);
      const TF ug = U[i][0] * Gm[0][j] + U[i][1] * Gm[1][j] + U[i][2] * Gm[2][j];
      L.C[q] = M[q] + cm * L.C[q] - cc * ug;
    }
}

// ------------------------------------------------------------------ record exchange
template <typename TF>
__device__ __forceinline__ void rec_shfl_down(Rec<TF> &dst, const Rec<TF> &src, int off,
                                              unsigned mask, int W) {
#pragma unroll
  for (int q = 0; q < 21; ++q) dst.C[q] = __shfl_down_sync(mask, src.C[q], off, W);
#pragma unroll
  for (int c = 0; c < 6; ++c) {
    dst.ds[c] = __shfl_down_sync(mask, src.ds[c], off, W);
    dst.tau[c] = __shfl_down_sync(mask, src.tau[c], off, W);
    dst.dd[c] = __shfl_down_sync(mask, src.dd[c], off, W);
  }
  dst.gg = __shfl_down_sync(mask, src.gg, off, W);
}

template <typename TF>
__device__ __forceinline__ void rec_store(double *slot, const Rec<TF> &r) {
#pragma unroll
  for (int q = 0; q < 21; ++q) slot[q] = double(r.C[q]);
#pragma unroll
  for (int c = 0; c < 6; ++c) {
    slot[21 + c] = double(r.ds[c]);
    slot[27 + c] = double(r.tau[c]);
    slot[33 + c] = double(r.dd[c]);
  }
  slot[39] = double(r.gg);
}

template <typename TF>
__device__ __forceinline__ void rec_load(Rec<TF> &r, const double *slot) {
#pragma unroll
  for (int q = 0; q < 21; ++q) r.C[q] = TF(slot[q]);
#pragma unroll
  for (int c = 0; c < 6; ++c) {
    r.ds[c] = TF(slot[21 + c]);
    r.tau[c] = TF(slot[27 + c]);
    r.dd[c] = TF(slot[33 + c]);
  }
  r.gg = TF(slot[39]);
}

}  // namespace dmn
