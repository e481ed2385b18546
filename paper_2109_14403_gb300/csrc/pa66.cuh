// pa66.cuh -- the PA66 matrix leaf (material kind 3) of arXiv 2109.14403,
// Sec. 4 (after Krairi et al.): a long-term branch C_inf and up to 12 Maxwell
// branches C_i with a common Poisson ratio, viscosities V_i = a_theta (3 K_i
// tau_K,i P1 + 2 G_i tau_G,i P2), tau_K,i = tau_i E_i / K_i, tau_G,i = tau_i E_i
// / G_i, the WLF shift log10 a_theta = -C1 (theta - theta_ref) / (C2 + theta -
// theta_ref), J2 viscoplasticity p_dot = (sigma_Y / eta) <(q - sigma_Y - H) /
// sigma_Y>^m with sigma_Y = Gamma1 sigma_Y0, H = Gamma1 k p^n, eta = Gamma2 eta0,
// Gamma_b = exp(-beta_b (theta - theta_ref)), and the model's coupling term
//   D = -theta (eps_dot - eps_vp_dot) : C_inf[alpha]
//       - theta sum_i (eps_dot - eps_vp_dot - eps_v,i_dot) : C_i[alpha]
//       + theta dH/dtheta p_dot + sigma_Y p_dot + sum_i sigma_v,i : eps_v,i_dot
// and dissipation sigma_Y p_dot + sum_i sigma_v,i : eps_v,i_dot.
//
// Implicit Euler makes every Maxwell branch linear in the leaf strain: with
// r = 1 / (1 + dt lambda), lambda_K = 1 / (a tau_K), lambda_G = 1 / (a tau_G),
// the branch strain at t^{n+1} is v + (1 - r)(e* - v) per projector, e* =
// eps - eps_vp - alpha (theta - theta0) I.  The leaf is therefore a J2
// viscoplastic law with effective moduli K_e = K_inf + sum K_i r_K,i, G_e =
// G_inf + sum G_i r_G,i and a history stress -3 h_v I - 2 h_d built from the
// branch strains at t^n; the branch sums the coupling term and its
// derivatives need (h, B, C, F, E below) are formed once per point from the
// 79 internal variables ("history", 34 words in shared memory), so a Newton
// pass costs no more than the Perzyna leaf's.  The branch strains themselves
// are updated once, after the last pass.
#pragma once
#include "dmn_kernels.cuh"

namespace dmn {

// history slots of a PA66 leaf (HP words):
//  0..5 eps_vp^n, 6 p^n, 7 3 h_v, 8..13 2 h_d, 14 S_v, 15 B_v, 16..21 B_d,
//  22 C_v, 23 C_d, 24 F_v, 25..30 F_d, 31 E_v, 32 E_d, 33 H(p^n)
// with v_i, d_i the mean and deviator of eps_v,i^n and
//  h_v = sum K_i r_K v_i, h_d = sum G_i r_G d_i, S_v = sum K_i (1 - r_K) v_i,
//  B = sum X_i r (1 - r) x_i, C = sum X_i r (1 - r) |x_i|^2,
//  F = sum X_i (1 - 2r) r (1 - r) x_i, E = sum X_i (1 - 2r) r (1 - r) |x_i|^2
//  (X = K, x = v for the volumetric sums; X = G, x = d for the deviatoric).
// Parked in the output state during the passes (8-byte slots of the leaf's
// z block): 0..5 eps_vp^{n+1}, 6 p^{n+1}, 7 mean of e*, 8..13 deviator of e*.

// per-point constants of a PA66 material
template <typename TF, typename HP>
struct MatPA {
  HP Ke3, G2e, G3e, KK, Kc3, Av, Ad, sy, c, Hk, a3th_idt, thb1, nh_h, idt;
  HP kr_v[kPaBranches], kr_d[kPaBranches], kq_v[kPaBranches], kq_d[kPaBranches];
  HP om_v[kPaBranches], om_d[kPaBranches], ko_v[kPaBranches];
  TF kf_v[kPaBranches], kf_d[kPaBranches];
  TF L, Avv, Add, Av_f, Ad_f, Ke_f, G2e_f, G3e_f, Kc_f, KK_f, sy_f, c_f, Hk_f, nh, b1, b2;
  TF alpha_f, theta_f, idt_f, a3th_idt_f;
  int m, nb;
  // static, per branch: K_i, G_i, K_i / (tau_i E_i), G_i / (tau_i E_i) (HP);
  // per material: K_inf, G_inf, sum K_i
  HP Kst[kPaBranches], Gst[kPaBranches], kvs[kPaBranches], gvs[kPaBranches];
  HP Kinf, Ginf, KKst;
};

template <typename T>
__device__ __forceinline__ T tpow(T x, T y);
template <>
__device__ __forceinline__ float tpow(float x, float y) { return powf(x, y); }
template <>
__device__ __forceinline__ double tpow(double x, double y) { return pow(x, y); }

// H = Hk p^n in FP64 (p > 0)
__device__ __forceinline__ double pa_hard(double Hk, double p, double n) {
  return p > 0.0 ? Hk * exp(n * log(p)) : 0.0;
}

// static constants of a PA66 material (once per CTA, FP64 then HP)
template <typename TF, typename HP>
__device__ void mat_static_pa(MatPA<TF, HP> &o, const MatDev &m) {
  HP *tag = nullptr;
  const double nu = m.pa[3];
  double KK = m.Kb;
  int nb = 0;
  for (int i = 0; i < kPaBranches; ++i) {
    const double Ei = m.pa[4 + i], tau = m.pa[16 + i];
    double Ki = 0.0, Gi = 0.0;
    if (Ei > 0.0) {
      nb = i + 1;
      Ki = Ei / (3.0 * (1.0 - 2.0 * nu));
      Gi = Ei / (2.0 * (1.0 + nu));
    }
    o.Kst[i] = hp_from(Ki, tag);
    o.Gst[i] = hp_from(Gi, tag);
    o.kvs[i] = hp_from(Ei > 0.0 ? Ki / (tau * Ei) : 0.0, tag);  // lambda_K = kvs / a
    o.gvs[i] = hp_from(Ei > 0.0 ? Gi / (tau * Ei) : 0.0, tag);  // lambda_G = gvs / a
    KK += Ki;
  }
  o.nb = nb;
  o.Kinf = hp_from(m.Kb, tag);
  o.Ginf = hp_from(m.G, tag);
  o.KKst = hp_from(KK, tag);
}

// the per-point constants, one thread per material: the WLF shift and the
// Gamma factors by FP64 exp, the branch factors r = 1 / (1 + dt lambda) and
// their sums in HP (no FP64 division per branch)
template <typename TF, typename HP>
__device__ void mat_point_pa(MatPA<TF, HP> &o, const MatDev &m, double theta, double dt) {
  HP *tag = nullptr;
  const double x = theta - m.pa[0], C1 = m.pa[1], C2 = m.pa[2];
  const double ln10 = 2.30258509299404568402;
  const double ia = exp(ln10 * C1 * x / (C2 + x));          // 1 / a_theta
  const double L = -ln10 * C1 * C2 / ((C2 + x) * (C2 + x));  // d ln a / d theta
  const double g1 = exp(-m.cE * x), g2 = exp(-m.pad_ * x);
  const double sy = g1 * m.sy0, eta = g2 * m.itv;
  const HP one = hp_from(1.0, tag), dtia = hp_from(dt * ia, tag);
  HP Ke = o.Kinf, Ge = o.Ginf, Kc = hp_zero(tag), Av = hp_zero(tag), Ad = hp_zero(tag);
  TF Avv = TF(0), Add = TF(0);
  for (int i = 0; i < kPaBranches; ++i) {
    if (i >= o.nb) {
      o.kr_v[i] = o.kr_d[i] = o.kq_v[i] = o.kq_d[i] = o.om_v[i] = o.om_d[i] = o.ko_v[i] = hp_zero(tag);
      o.kf_v[i] = o.kf_d[i] = TF(0);
      continue;
    }
    const HP tv = dtia * o.kvs[i], td = dtia * o.gvs[i];  // dt lambda
    const HP rv = hp_div(one, one + tv), rd = hp_div(one, one + td);
    const HP omv = tv * rv, omd = td * rd;                  // 1 - r without cancellation
    const HP Ki = o.Kst[i], Gi = o.Gst[i];
    o.kr_v[i] = Ki * rv;
    o.kr_d[i] = Gi * rd;
    o.kq_v[i] = o.kr_v[i] * omv;
    o.kq_d[i] = o.kr_d[i] * omd;
    o.om_v[i] = omv;
    o.om_d[i] = omd;
    o.ko_v[i] = Ki * omv;
    const TF rvf = tf_of(rv, (TF *)nullptr), rdf = tf_of(rd, (TF *)nullptr);
    o.kf_v[i] = (TF(1) - TF(2) * rvf) * tf_of(o.kq_v[i], (TF *)nullptr);
    o.kf_d[i] = (TF(1) - TF(2) * rdf) * tf_of(o.kq_d[i], (TF *)nullptr);
    Ke = Ke + o.kr_v[i];
    Ge = Ge + o.kr_d[i];
    Kc = Kc + o.ko_v[i];
    Av = Av + o.kq_v[i];
    Ad = Ad + o.kq_d[i];
    Avv += o.kf_v[i];
    Add += o.kf_d[i];
  }
  const HP three = hp_from(3.0, tag), two = hp_from(2.0, tag);
  o.Ke3 = three * Ke;
  o.G2e = two * Ge;
  o.G3e = three * Ge;
  o.KK = o.KKst;
  o.Kc3 = three * Kc;
  o.Av = Av;
  o.Ad = Ad;
  o.sy = hp_from(sy, tag);
  o.c = hp_from(dt * sy / eta, tag);
  o.Hk = hp_from(g1 * m.dsy, tag);
  o.a3th_idt = hp_from(3.0 * m.alpha * theta / dt, tag);
  o.thb1 = hp_from(theta * m.cE, tag);
  o.nh_h = hp_from(m.H, tag);
  o.idt = hp_from(1.0 / dt, tag);
  o.L = TF(L);
  o.Avv = Avv;
  o.Add = Add;
  o.Av_f = tf_of(Av, (TF *)nullptr);
  o.Ad_f = tf_of(Ad, (TF *)nullptr);
  o.Ke_f = tf_of(Ke, (TF *)nullptr);
  o.G2e_f = tf_of(o.G2e, (TF *)nullptr);
  o.G3e_f = tf_of(o.G3e, (TF *)nullptr);
  o.Kc_f = tf_of(Kc, (TF *)nullptr);
  o.KK_f = tf_of(o.KK, (TF *)nullptr);
  o.sy_f = TF(sy);
  o.c_f = TF(dt * sy / eta);
  o.Hk_f = TF(g1 * m.dsy);
  o.nh = TF(m.H);
  o.b1 = TF(m.cE);
  o.b2 = TF(m.pad_);
  o.alpha_f = TF(m.alpha);
  o.theta_f = TF(theta);
  o.idt_f = TF(1.0 / dt);
  o.a3th_idt_f = TF(3.0 * m.alpha * theta / dt);
  o.m = int(m.mexp + 0.5);
}

// history of one PA66 leaf from its internal variables at t^n (FP64, state)
template <typename TF, typename HP>
__device__ void pa_history(const MatPA<TF, HP> &m, const double *zn, HP *h) {
  HP *tag = nullptr;
#pragma unroll
  for (int c = 0; c < 7; ++c) h[c] = hp_load(zn[c], tag);
  const HP third = hp_from(1.0 / 3.0, tag);
  HP hv = hp_zero(tag), Sv = hp_zero(tag), Bv = hp_zero(tag), Cv = hp_zero(tag), Cd = hp_zero(tag);
  HP hd[6], Bd[6];
  TF Fd[6], Fv = TF(0), Ev = TF(0), Ed = TF(0);
#pragma unroll
  for (int c = 0; c < 6; ++c) {
    hd[c] = hp_zero(tag);
    Bd[c] = hp_zero(tag);
    Fd[c] = TF(0);
  }
  for (int i = 0; i < m.nb; ++i) {
    const double *z = zn + 7 + 6 * i;
    HP e[6];
#pragma unroll
    for (int c = 0; c < 6; ++c) e[c] = hp_load(z[c], tag);
    const HP v = (e[0] + e[1] + e[2]) * third;
    HP d[6];
#pragma unroll
    for (int c = 0; c < 6; ++c) d[c] = c < 3 ? e[c] - v : e[c];
    HP dd = d[0] * d[0];
#pragma unroll
    for (int c = 1; c < 6; ++c) dd = dd + d[c] * d[c];
    hv = hv + m.kr_v[i] * v;
    Sv = Sv + m.ko_v[i] * v;
    Bv = Bv + m.kq_v[i] * v;
    Cv = Cv + m.kq_v[i] * (v * v);
    Cd = Cd + m.kq_d[i] * dd;
    const TF vf = tf_of(v, (TF *)nullptr);
    Fv += m.kf_v[i] * vf;
    Ev += m.kf_v[i] * vf * vf;
    Ed += m.kf_d[i] * tf_of(dd, (TF *)nullptr);
#pragma unroll
    for (int c = 0; c < 6; ++c) {
      hd[c] = hd[c] + m.kr_d[i] * d[c];
      Bd[c] = Bd[c] + m.kq_d[i] * d[c];
      Fd[c] += m.kf_d[i] * tf_of(d[c], (TF *)nullptr);
    }
  }
  h[7] = hv + hv + hv;
#pragma unroll
  for (int c = 0; c < 6; ++c) {
    h[8 + c] = hd[c] + hd[c];
    h[16 + c] = Bd[c];
    h[25 + c] = hp_add_tf(hp_zero(tag), Fd[c]);
  }
  h[14] = Sv;
  h[15] = Bv;
  h[22] = Cv;
  h[23] = Cd;
  h[24] = hp_add_tf(hp_zero(tag), Fv);
  h[31] = hp_add_tf(hp_zero(tag), Ev);
  h[32] = hp_add_tf(hp_zero(tag), Ed);
  h[33] = hp_from(pa_hard(hp_to(m.Hk), zn[6], hp_to(m.nh_h)), tag);
}

// One pass of the PA66 leaf at strain eps: stress, D and dissipation in HP,
// derivatives into the TF record; parks eps_vp, p and e* in zp.
template <typename TF, typename HP>
__device__ __forceinline__ void leaf_pa66(const MatPt<TF, HP> &mp, const MatPA<TF, HP> &m,
                                          const HP eps[6], const HP *h, HP trn, HP sig[6], HP &D,
                                          HP &X, Rec<TF> &R, HP *zp) {
  HP *tag = nullptr;
  const TF S32 = TF(1.2247448713915890491);  // sqrt(3/2)
  const HP ev = (eps[0] + eps[1] + eps[2]) * mp.third;
  const HP esv = ev - mp.ath;  // mean of e*
  HP dv[6], s[6];              // dev eps - eps_vp^n; trial deviator
#pragma unroll
  for (int c = 0; c < 6; ++c) {
    dv[c] = (c < 3 ? eps[c] - ev : eps[c]) - h[c];
    s[c] = m.G2e * dv[c] - h[8 + c];
  }
  const HP sm = m.Ke3 * esv - h[7];  // mean stress
  HP sn2 = s[0] * s[0];
#pragma unroll
  for (int c = 1; c < 6; ++c) sn2 = sn2 + s[c] * s[c];
  const HP q2 = mp.c15 * sn2;
  const HP yr = m.sy + h[33];
  const bool plastic = hp_gt(q2, yr * yr);
  HP dp = hp_zero(tag), kap = hp_zero(tag), R1 = h[33];
  TF kinv = TF(0), rho = TF(0), phif = TF(0), Rp1 = TF(0), qf = TF(0);
  TF Nf[6] = {TF(0), TF(0), TF(0), TF(0), TF(0), TF(0)};
  const TF pnf = tf_of(h[6], (TF *)nullptr);
  if (plastic) {
    const HP q = hp_sqrt(q2);
    qf = tf_of(q, (TF *)nullptr);
    const TF isy = TF(1) / m.sy_f, G3 = m.G3e_f, cf = m.c_f;
    const int me = m.m;
    // safeguarded Newton on g(x) = x - c phi(x)^m in TF, bracket [0, f / 3G_e]
    TF lo = TF(0), hi = (qf - m.sy_f - tf_of(h[33], (TF *)nullptr)) / G3, x = TF(0), gp = TF(1);
    if (hi < TF(0)) hi = TF(0);
    for (int it = 0; it < 80; ++it) {
      const TF p1 = pnf + x;
      const TF Rr = p1 > TF(0) ? m.Hk_f * tpow(p1, m.nh) : TF(0);
      const TF Rp = p1 > TF(0) ? m.nh * Rr / p1 : TF(1e30);
      TF phi = (qf - G3 * x - m.sy_f - Rr) * isy;
      if (phi < TF(0)) phi = TF(0);
      TF pw = TF(1);
      for (int k = 1; k < me; ++k) pw *= phi;
      const TF gx = x - cf * pw * phi;
      if (gx < TF(0)) lo = x;
      else hi = x;
      gp = TF(1) + cf * TF(me) * pw * (G3 + Rp) * isy;
      TF xn = x - gx / gp;
      if (!(xn > lo && xn < hi)) xn = TF(0.5) * (lo + hi);
      const TF step = fabs(xn - x);
      x = xn;
      if (!(step > TF(sizeof(TF) == 4 ? 1e-7 : 1e-15) * x) || !(hi - lo > TF(sizeof(TF) == 4 ? 1e-7 : 1e-15) * hi))
        break;
    }
    // two corrections in HP; H linearised about x with an FP64 value there
    const double p0 = hp_to(h[6]) + double(x);
    const HP R0 = hp_from(pa_hard(hp_to(m.Hk), p0, hp_to(m.nh_h)), tag);
    const TF Rp0 = p0 > 0.0 ? m.nh * tf_of(R0, (TF *)nullptr) / TF(p0) : TF(0);
    {
      const TF p1 = pnf + x;
      TF phi = (qf - G3 * x - m.sy_f - tf_of(R0, (TF *)nullptr)) * isy;
      if (phi < TF(0)) phi = TF(0);
      TF pw = TF(1);
      for (int k = 1; k < me; ++k) pw *= phi;
      gp = TF(1) + cf * TF(me) * pw * (G3 + (p1 > TF(0) ? Rp0 : TF(0))) * isy;
    }
    const TF igp = TF(1) / gp;
    const HP isyh = hp_div(mp.one, m.sy);
    dp = hp_add_tf(hp_zero(tag), x);
    for (int k2 = 0; k2 < 2; ++k2) {
      const HP Rd = R0 + (dp - hp_add_tf(hp_zero(tag), x)) * Rp0;
      HP ph = (q - m.G3e * dp - m.sy - Rd) * isyh;
      if (tf_of(ph, (TF *)nullptr) < TF(0)) ph = hp_zero(tag);
      HP pwm = ph;
      for (int k = 1; k < me; ++k) pwm = pwm * ph;
      const HP g = dp - m.c * pwm;
      dp = dp - g * igp;
    }
    R1 = R0 + (dp - hp_add_tf(hp_zero(tag), x)) * Rp0;
    phif = tf_of((q - m.G3e * dp - m.sy - R1) * isyh, (TF *)nullptr);
    if (phif < TF(0)) phif = TF(0);
    TF pw = TF(1);
    for (int k = 1; k < me; ++k) pw *= phif;
    const TF cm = cf * TF(me) * pw;
    const TF p1f = pnf + tf_of(dp, (TF *)nullptr);
    Rp1 = p1f > TF(0) ? m.nh * tf_of(R1, (TF *)nullptr) / p1f : TF(0);
    const TF den = m.sy_f + cm * (G3 + Rp1);
    kinv = cm / den;
    rho = m.sy_f / den;
    kap = hp_div(dp, q);
    const TF isn = TF(1) / sqrt(tf_of(sn2, (TF *)nullptr));
#pragma unroll
    for (int c = 0; c < 6; ++c) Nf[c] = tf_of(s[c], (TF *)nullptr) * isn;
  }
  // stress, updated viscoplastic strain, e*
  const HP th1h = mp.one - m.G3e * kap, kz = mp.c15 * kap;
  HP esd[6];
#pragma unroll
  for (int c = 0; c < 6; ++c) {
    const HP dvp = kz * s[c];  // d eps_vp
    sig[c] = c < 3 ? sm + th1h * s[c] : th1h * s[c];
    zp[c] = h[c] + dvp;
    esd[c] = dv[c] - dvp;
  }
  zp[6] = h[6] + dp;
  zp[7] = esv;
#pragma unroll
  for (int c = 0; c < 6; ++c) zp[8 + c] = esd[c];
  // coupling term and dissipation
  const HP trde = (eps[0] + eps[1] + eps[2]) - trn;
  const HP T1 = m.KK * trde - m.Kc3 * esv + (h[14] + h[14] + h[14]);
  HP dmv = esv * (m.Av * esv - (h[15] + h[15])) + h[22];
  HP dmd = h[23];
#pragma unroll
  for (int c = 0; c < 6; ++c) dmd = dmd + esd[c] * (m.Ad * esd[c] - (h[16 + c] + h[16 + c]));
  const HP dmx = (dmv * hp_from(9.0, tag) + (dmd + dmd)) * m.idt;
  const HP dsy = m.sy * dp * m.idt;
  X = dsy + dmx;
  D = (dsy - m.thb1 * R1 * dp * m.idt) + dmx - m.a3th_idt * T1;
  // ---- derivatives (TF) ----
  const TF kapf = tf_of(kap, (TF *)nullptr), dpf = tf_of(dp, (TF *)nullptr);
  const TF G2 = m.G2e_f, G3 = m.G3e_f;
  const TF th1 = TF(1) - G3 * kapf;
  const TF thb = plastic ? G3 * (kinv - kapf) : TF(0);
  const TF cP1 = m.Ke_f - G2 * th1 / TF(3), cI = G2 * th1, cN = G2 * thb;
#pragma unroll
  for (int i = 0; i < 6; ++i)
#pragma unroll
    for (int j = i; j < 6; ++j)
      R.C[sidx(i, j)] = (i < 3 && j < 3 ? cP1 : TF(0)) + (i == j ? cI : TF(0)) - cN * Nf[i] * Nf[j];
  const TF L = m.L, idt = m.idt_f, al = m.alpha_f, th = m.theta_f, b1 = m.b1;
  const TF esvf = tf_of(esv, (TF *)nullptr);
  const TF Bvf = tf_of(h[15], (TF *)nullptr);
  const TF wv = m.Av_f * esvf - Bvf;
  // d sigma / d theta
  TF ttr[6], sf[6], wf[6], esdf[6];
  TF Nt = TF(0), Nw = TF(0);
#pragma unroll
  for (int c = 0; c < 6; ++c) {
    ttr[c] = TF(2) * L * (m.Ad_f * tf_of(dv[c], (TF *)nullptr) - tf_of(h[16 + c], (TF *)nullptr));
    sf[c] = tf_of(s[c], (TF *)nullptr);
    esdf[c] = tf_of(esd[c], (TF *)nullptr);
    wf[c] = m.Ad_f * esdf[c] - tf_of(h[16 + c], (TF *)nullptr);
    Nt += Nf[c] * ttr[c];
    Nw += Nf[c] * wf[c];
  }
  const TF Rf = tf_of(R1, (TF *)nullptr);
  TF ddp = TF(0), dth1 = TF(0);
  if (plastic) {
    const TF dqtr = S32 * Nt;
    ddp = rho * (m.b2 - b1) * dpf +
          kinv * (dqtr - TF(3) * L * m.Ad_f * dpf + b1 * m.sy_f * (TF(1) + phif) + b1 * Rf);
    dth1 = -TF(3) * L * m.Ad_f * kapf - G3 * (ddp - kapf * dqtr) / qf;
  }
  const TF taum = TF(3) * L * wv - TF(3) * m.Ke_f * al;
#pragma unroll
  for (int c = 0; c < 6; ++c) R.tau[c] = (c < 3 ? taum : TF(0)) + th1 * ttr[c] + dth1 * sf[c];
  // d D / d eps
  const TF dDp = plastic ? (m.sy_f - th * b1 * (Rf + Rp1 * dpf)) * kinv * S32 * G2 * idt : TF(0);
  const TF dth = -m.a3th_idt_f * m.Ke_f;
#pragma unroll
  for (int c = 0; c < 6; ++c)
    R.dd[c] = (c < 3 ? dth + TF(6) * wv * idt : TF(0)) + dDp * Nf[c] +
              TF(4) * (th1 * wf[c] - thb * Nw * Nf[c]) * idt;
  // d D / d theta
  const TF T1f = tf_of(T1, (TF *)nullptr);
  const TF dT1 = TF(3) * L * m.Av_f * esvf + TF(3) * m.Kc_f * al - TF(3) * L * Bvf;
  TF gg = -TF(3) * al * T1f * idt - m.a3th_idt_f * dT1;
  if (plastic)
    gg += ((-b1 * m.sy_f - b1 * Rf + th * b1 * b1 * Rf) * dpf +
           (m.sy_f - th * b1 * Rf - th * b1 * Rp1 * dpf) * ddp) * idt;
  // de*' / d theta = -d eps_vp / d theta
  TF wde = TF(0), e2 = TF(0), eF = TF(0);
#pragma unroll
  for (int c = 0; c < 6; ++c) {
    const TF devp = plastic ? S32 * ddp * Nf[c] + TF(1.5) * kapf * (ttr[c] - Nt * Nf[c]) : TF(0);
    wde -= wf[c] * devp;
    e2 += esdf[c] * esdf[c];
    eF += esdf[c] * tf_of(h[25 + c], (TF *)nullptr);
  }
  const TF Fvf = tf_of(h[24], (TF *)nullptr), Evf = tf_of(h[31], (TF *)nullptr),
           Edf = tf_of(h[32], (TF *)nullptr);
  gg += (TF(9) * (L * (m.Avv * esvf * esvf - TF(2) * esvf * Fvf + Evf) - TF(2) * al * wv) +
         TF(2) * (L * (m.Add * e2 - TF(2) * eF + Edf) + TF(2) * wde)) * idt;
  R.gg = gg;
#pragma unroll
  for (int c = 0; c < 6; ++c) R.ds[c] = TF(0);
}

// after the last pass: the leaf's internal variables at t^{n+1} (FP64) from
// the parked eps_vp, p, e* and the branch strains at t^n
template <typename TF, typename HP>
__device__ void pa_finish(const MatPA<TF, HP> &m, const double *zn, double *zo) {
  HP *tag = nullptr;
  const HP *zp = reinterpret_cast<const HP *>(zo);
  HP par[14];
#pragma unroll
  for (int c = 0; c < 14; ++c) par[c] = zp[c];
  const HP third = hp_from(1.0 / 3.0, tag);
  for (int i = 0; i < kPaBranches; ++i) {
    const double *z = zn + 7 + 6 * i;
    double *o = zo + 7 + 6 * i;
    if (i >= m.nb) {
      for (int c = 0; c < 6; ++c) o[c] = z[c];
      continue;
    }
    HP e[6];
#pragma unroll
    for (int c = 0; c < 6; ++c) e[c] = hp_load(z[c], tag);
    const HP v = (e[0] + e[1] + e[2]) * third;
    const HP vn = v + m.om_v[i] * (par[7] - v);
#pragma unroll
    for (int c = 0; c < 6; ++c) {
      const HP d = c < 3 ? e[c] - v : e[c];
      const HP dn = d + m.om_d[i] * (par[8 + c] - d);
      o[c] = hp_to(c < 3 ? dn + vn : dn);
    }
  }
#pragma unroll
  for (int c = 0; c < 7; ++c) zo[c] = hp_to(par[c]);
}

}  // namespace dmn
