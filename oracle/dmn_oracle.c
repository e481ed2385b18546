/*
 * dmn_oracle.c -- plain, slow FP64 CPU reference of the online evaluation of a
 * thermomechanical direct deep material network (Gajek, Schneider, Boehlke,
 * "An FE-DMN method for the multiscale analysis of thermomechanical composites",
 * arXiv 2109.14403, Section 3.3 and Algorithm 1).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link or call this
 * file: only the test suite, the package's smoke check and the CPU-baseline leg
 * of the benchmark use it.  It shares no code, header or constant with the CUDA
 * library; the state layout it reads and writes is the documented interface of
 * that library, re-implemented here from its description.
 *
 * What it computes (all in FP64):
 *  - Section 3.1: weight propagation w^i_k = w^{2i-1}_{k+1} + w^{2i}_{k+1}, the
 *    volume fractions c_{k,1}, c_{k,2}, and the ordering of the lamination
 *    directions (bottom level first, root last).
 *  - Eq. (DMN kinematics): leaf strains eps = eps_bar + A a with an EXPLICIT
 *    operator A.  The paper defers the form of A to Gajek et al. (2020); the
 *    reading used here: for a node p with children 1 and 2 and jump a_p, every
 *    leaf under child 1 receives +c_{p,2} sym(a_p (x) n_p) and every leaf under
 *    child 2 receives -c_{p,1} sym(a_p (x) n_p).  The weighted mean strain of a
 *    node then equals its parent's, and the strain jump across node p equals
 *    sym(a_p (x) n_p).
 *  - Eq. (Euler-Lagrange) residual A^T W sigma, eq. (Newton) Hessian
 *    A^T W dsigma/deps A, assembled block by block; block (p,q) is non-zero only
 *    when p and q lie on one root-leaf path.
 *  - The Hessian is factored by a block Cholesky that eliminates the nodes in
 *    the paper's order (bottom level first, root last); every node's column
 *    only touches its ancestors, which already form a dense block, so there is
 *    no fill.  For small K a second path forms a dense A, a dense Hessian and a
 *    dense Cholesky; the two must agree to rounding.
 *  - Algorithm 1 step by step: warm start a <- a^n, Residual, Newton solve,
 *    Backtracking with gamma^i (1 - gamma), break on res < tol.
 *  - Eqs. (effective stress, coupling term, dissipation) and the four
 *    algorithmic tangents via the linear systems for da/deps_bar and
 *    da/dtheta (seven right-hand sides re-using the factor), then
 *    eqs. (ddsdde, ddsddt, drplde, drpldt).
 *
 * Phase laws:
 *  - kind 0, isotropic linear thermoelastic (Section 4, E-glass):
 *      sigma = C[eps - alpha (theta - theta0) I], C = 3K P1 + 2G P2,
 *      D = -theta eps_dot : C[alpha], dissipation 0.
 *  - kind 1, J2 elastoplastic with linear isotropic hardening H and a yield
 *    stress falling linearly with temperature (the rate-independent special
 *    case of the J2 flow rule of Section 4 with psi_mech of eq. (PA66 psi)
 *    restricted to one elastic branch and hardening energy H p^2 / 2).
 *    Implicit Euler of Biot's equation = radial return with the closed-form
 *    plastic multiplier dp = f_trial / (3G + H).
 *    Coupling term and dissipation are the discrete forms of the paper's
 *    D = theta d2psi/dtheta deps : eps_dot + theta d2psi/dtheta dz . z_dot
 *        - dpsi/dz . z_dot, i.e.
 *      D = [-3 K alpha theta tr(eps - eps^n) + sigma_Y(theta) dp] / dt,
 *      Diss = sigma_Y(theta) dp / dt.
 *  - kind 2, J2 viscoplasticity of Perzyna (overstress) type with the
 *    accumulated plastic strain rate of Section 4 (eq. for p_dot of the PA66
 *    model, with linear hardening H p and the reading sigma_Y / eta = 1 / t_visc),
 *      p_dot = (1 / t_visc) < (q - sigma_Y(theta) - H p) / sigma_Y(theta) >_+^m,
 *    and temperature-dependent moduli E(theta) = E (1 + dE_dT (theta - theta0)).
 *    Implicit Euler: dp solves dp = (dt / t_visc) phi^m with
 *    phi = (q_trial - (3G + H) dp - sigma_Y - H p^n) / sigma_Y (scalar Newton,
 *    kept inside [0, f_trial / (3G + H)]).  The consistent tangent is the
 *    radial-return one with H replaced by H + h_v, h_v = sigma_Y / (c m phi^(m-1)),
 *    c = dt / t_visc.  With C(theta) = r(theta) C0 the paper's coupling term gains
 *    theta dC/dtheta eps_e : (eps_dot - eps_p_dot) (from d2psi/dtheta deps and
 *    d2psi/dtheta deps_p), so
 *      D = [theta (r'/r) sigma : (de - deps_p) - 3 K alpha theta tr(de)
 *           + sigma_Y dp] / dt,   Diss = sigma_Y dp / dt,
 *    with de = eps - eps^n the leaf's strain increment; the leaf keeps its
 *    strain in its internal variables: z = (eps_p (6), p, eps (6)).
 *  - kind 3, the PA66 matrix of Section 4 (after Krairi et al.): eq. (PA66 psi)
 *    with a long-term branch C_inf and N <= 12 Maxwell branches C_i (constant
 *    nu), thermorheologically simple viscosities V_i = a_theta (3 K_i tau_K,i P1
 *    + 2 G_i tau_G,i P2), tau_K,i = tau_i E_i / K_i, tau_G,i = tau_i E_i / G_i,
 *    WLF shift log10 a_theta = -C1 (theta - theta_ref) / (C2 + theta - theta_ref),
 *    J2 viscoplasticity with p_dot = (sigma_Y / eta) <(q - sigma_Y - H) / sigma_Y>_+^m,
 *    sigma_Y = Gamma(theta, beta1) sigma_Y0, H = Gamma(theta, beta1) k p^n,
 *    eta = Gamma(theta, beta2) eta0, Gamma = exp(-beta (theta - theta_ref)), and the
 *    coupling term D and dissipation of the PA66 model.  Every evolution equation
 *    is integrated by implicit Euler; for a trial dp the viscoplastic strain moves
 *    along the trial deviator (the flow direction of the J2 law), every Maxwell
 *    strain is updated in closed form, the stress is summed over the branches,
 *    and dp is found by bisection of dp = dt p_dot(dp).  Rates in D are
 *    (x^{n+1} - x^n) / dt.  The derivatives d sigma/d eps, d sigma/d theta,
 *    dD/d eps and dD/d theta are taken by the complex-step method (Squire and
 *    Trapp 1998): the law is evaluated in complex arithmetic with one input
 *    perturbed by i h, and the derivative is Im(out) / h, exact to rounding;
 *    dp is carried into the complex plane by Newton steps on the same equation.
 *    z = (eps_vp (6), p, eps_v,1 (6), ..., eps_v,12 (6)): 79 words.
 *
 * Symmetric tensors are Mandel 6-vectors (11, 22, 33, sqrt2*23, sqrt2*13,
 * sqrt2*12); fourth-order tensors are 6x6 matrices acting on them.
 *
 * Readings where the paper is silent (each also listed in the design notes):
 *  - relative residual denominator: max(|sigma_bar|_F, res_floor);
 *  - maxit, maxbacktrack, gamma are parameters (defaults 50, 8, 0.5);
 *  - sigma_Y(theta) = sy0 + dsy_dT (theta - theta0), floored at 1e-6 MPa;
 *  - zero leaf weights are rejected (the Hessian would be singular).
 *
 * The test suite pins this code against closed-form laminates, homogeneous
 * phases, free thermal expansion, Hill-Mandel, finite-difference tangents and
 * dense-versus-sparse agreement.  A full inelastic K=8 path is pinned by
 * composition: leaf strains by the kinematics, leaf responses by the pinned
 * leaf law, equilibrium of the converged jumps by virtual work.  The paper
 * prints no worked example to compare values with.
 */
#include <complex.h>
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_SQ2 1.41421356237309504880
#define OR_MAXK 10

/* ------------------------------------------------------------------ */
/* tree                                                                 */
/* ------------------------------------------------------------------ */

/* material row, 40 words:
   kinds 0-2: kind E nu alpha theta0 sy0 dsy_dT H m t_visc dE_dT, then 0
   kind 3:    kind E_inf nu alpha0 theta0 sy0 k n m eta0 beta1 beta2 theta_ref C1 C2 0,
              E_1..E_12, tau_1..tau_12 */
#define OR_MATW 40
#define OR_NMAX 12 /* Maxwell branches of kind 3 */
#define OR_ZMAX 79 /* internal variables per leaf, at most */

typedef struct {
  int kind;
  double E, nu, alpha, theta0, sy0, dsy_dT, H;
  double m_rate, t_visc, dE_dT; /* kind 2 only */
  double row[OR_MATW];          /* the row as given */
} omat;

/* words of internal variables of a leaf of this kind */
static int z_words(int kind) {
  return kind == 1 ? 7 : (kind == 2 ? 13 : (kind == 3 ? 7 + 6 * OR_NMAX : 0));
}

typedef struct {
  int K, nleaf, nnode;
  double w[1 << OR_MAXK];            /* leaf weights, leaf j = 0..2^K-1   */
  double n[(1 << OR_MAXK)][3];       /* normals, paper order              */
  double c1[(1 << OR_MAXK)], c2[(1 << OR_MAXK)];
  int depth[(1 << OR_MAXK)];         /* level k of node (1 = root)        */
  /* for each leaf j and level k = 1..K: ancestor node index and sign s  */
  int anc[1 << OR_MAXK][OR_MAXK];
  double s[1 << OR_MAXK][OR_MAXK];
  int phase[1 << OR_MAXK];
  int zoff[1 << OR_MAXK];            /* offset of the leaf's z in state   */
  int state_words;
} otree;

/* paper index of node (level k, position i), 1-based k and i */
static int pidx(int K, int k, int i) { return (1 << K) - (1 << k) + (i - 1); }

static int build_tree(otree *t, int K, const double *leaf_w, const double *normals,
                      const uint8_t *phase, const omat *mats, int n_mats) {
  if (K < 1 || K > OR_MAXK) return -1;
  t->K = K;
  t->nleaf = 1 << K;
  t->nnode = (1 << K) - 1;
  double wsum = 0.0;
  for (int j = 0; j < t->nleaf; ++j) {
    if (!(leaf_w[j] > 0.0)) return -2;
    t->w[j] = leaf_w[j];
    wsum += leaf_w[j];
    if (phase[j] >= n_mats) return -3;
    t->phase[j] = phase[j];
  }
  if (fabs(wsum - 1.0) > 1e-12) return -4;
  for (int p = 0; p < t->nnode; ++p) {
    double nn = sqrt(normals[3 * p] * normals[3 * p] + normals[3 * p + 1] * normals[3 * p + 1] +
                     normals[3 * p + 2] * normals[3 * p + 2]);
    if (!(nn > 0.0)) return -5;
    for (int c = 0; c < 3; ++c) t->n[p][c] = normals[3 * p + c] / nn;
  }
  /* weight propagation (Section 3.1): level K+1 = leaves */
  double wl[OR_MAXK + 2][1 << OR_MAXK];
  for (int j = 0; j < t->nleaf; ++j) wl[K + 1][j] = t->w[j];
  for (int k = K; k >= 1; --k) {
    for (int i = 1; i <= (1 << (k - 1)); ++i) {
      double wa = wl[k + 1][2 * i - 2], wb = wl[k + 1][2 * i - 1];
      wl[k][i - 1] = wa + wb;
      int p = pidx(K, k, i);
      t->c1[p] = wa / (wa + wb);
      t->c2[p] = 1.0 - t->c1[p];
      t->depth[p] = k;
    }
  }
  /* explicit kinematic operator: ancestors and signs of every leaf */
  for (int j = 0; j < t->nleaf; ++j) {
    for (int k = 1; k <= K; ++k) {
      int i = (j >> (K + 1 - k)) + 1;              /* ancestor position at level k */
      int p = pidx(K, k, i);
      int first_child = ((j >> (K - k)) & 1) == 0; /* under child 2i-1 ?          */
      t->anc[j][k - 1] = p;
      t->s[j][k - 1] = first_child ? t->c2[p] : -t->c1[p];
    }
  }
  int off = 8 + 3 * t->nnode;
  for (int j = 0; j < t->nleaf; ++j) {
    const int zw = z_words(mats[t->phase[j]].kind);
    if (zw > 0) {
      t->zoff[j] = off;
      off += zw;
    } else {
      t->zoff[j] = -1;
    }
  }
  if (off & 1) off += 1;
  t->state_words = off;
  return 0;
}

/* B_p a = sym(a (x) n_p) as a Mandel vector; B is 6x3 */
static void bmat(const double n[3], double B[6][3]) {
  memset(B, 0, sizeof(double) * 18);
  const double r = 1.0 / OR_SQ2;
  B[0][0] = n[0];
  B[1][1] = n[1];
  B[2][2] = n[2];
  B[3][1] = r * n[2]; B[3][2] = r * n[1];
  B[4][0] = r * n[2]; B[4][2] = r * n[0];
  B[5][0] = r * n[1]; B[5][1] = r * n[0];
}

/* ------------------------------------------------------------------ */
/* phase laws                                                           */
/* ------------------------------------------------------------------ */

typedef struct {
  double sig[6];    /* stress                                 */
  double C[6][6];   /* dsigma/deps                            */
  double tau[6];    /* dsigma/dtheta                          */
  double D;         /* coupling term D_i                      */
  double d[6];      /* dD/deps                                */
  double g;         /* dD/dtheta (explicit)                   */
  double diss;      /* dissipation                            */
  double znew[OR_ZMAX]; /* eps_p (6), p [, eps (6) for kind 2; Maxwell strains for kind 3] */
} oleaf;

static const double M1[6] = {1, 1, 1, 0, 0, 0};

/* ------------------------------------------------------------ kind 3: PA66 */

typedef double complex ocx;

typedef struct {
  double Einf, nu, alpha, theta0, sy0, k, n, m, eta0, beta1, beta2, theta_ref, C1, C2;
  double Ei[OR_NMAX], taui[OR_NMAX];
} opa66;

static void pa66_params(const double *r, opa66 *P) {
  P->Einf = r[1]; P->nu = r[2]; P->alpha = r[3]; P->theta0 = r[4]; P->sy0 = r[5];
  P->k = r[6]; P->n = r[7]; P->m = r[8]; P->eta0 = r[9]; P->beta1 = r[10]; P->beta2 = r[11];
  P->theta_ref = r[12]; P->C1 = r[13]; P->C2 = r[14];
  for (int i = 0; i < OR_NMAX; ++i) { P->Ei[i] = r[16 + i]; P->taui[i] = r[28 + i]; }
}

/* everything the PA66 law returns for one (complex) input */
typedef struct {
  ocx sig[6], D, diss, znew[OR_ZMAX];
} opa66_out;

/* mean and deviator of a Mandel vector: x = mean m + dev */
static void split(const ocx x[6], ocx *mean, ocx dev[6]) {
  *mean = (x[0] + x[1] + x[2]) / 3.0;
  for (int c = 0; c < 6; ++c) dev[c] = x[c] - M1[c] * (*mean);
}

/* The law at strain eps and temperature theta with the viscoplastic increment
   dp given: eps_vp = eps_vp^n + dp (3/2) N_tr / |N_tr| sqrt(2/3)... i.e. along
   the unit trial deviator ntr (d eps_vp = sqrt(3/2) dp ntr); the Maxwell strains
   follow by implicit Euler.  Returns q = sqrt(3/2) |dev sigma| in *q and fills
   out (stress, D, dissipation, new internal variables). */
static void pa66_at(const opa66 *P, const ocx eps[6], ocx theta, const double *zn, double trn,
                    double dt, ocx dp, const ocx ntr[6], ocx *q, opa66_out *o) {
  const ocx x = theta - P->theta_ref;
  const ocx a = cpow(10.0, -P->C1 * x / (P->C2 + x));       /* WLF shift a_theta */
  const ocx G1 = cexp(-P->beta1 * x), G2 = cexp(-P->beta2 * x);
  const ocx sy = G1 * P->sy0;
  const double Kinf = P->Einf / (3.0 * (1.0 - 2.0 * P->nu)), Ginf = P->Einf / (2.0 * (1.0 + P->nu));
  ocx evp[6], es[6];
  for (int c = 0; c < 6; ++c) {
    evp[c] = zn[c] + sqrt(1.5) * dp * ntr[c];
    es[c] = eps[c] - evp[c] - M1[c] * P->alpha * (theta - P->theta0); /* eps - eps_vp - alpha dtheta I */
  }
  ocx es_m, es_d[6];
  split(es, &es_m, es_d);
  /* long-term branch */
  ocx sig[6];
  for (int c = 0; c < 6; ++c) sig[c] = 3.0 * Kinf * es_m * M1[c] + 2.0 * Ginf * es_d[c];
  /* Maxwell branches: d eps_v / dt = F_i sigma_v,i, F_i the pseudo-inverse of V_i */
  ocx trdev_sum = 0.0; /* sum_i 3 K_i alpha tr(d eps - d eps_v,i) */
  ocx visc = 0.0;      /* sum_i sigma_v,i : d eps_v,i */
  const double treps_n = trn;
  const ocx treps = eps[0] + eps[1] + eps[2];
  for (int i = 0; i < OR_NMAX; ++i) {
    const double *vn = zn + 7 + 6 * i;
    ocx *vnew = o->znew + 7 + 6 * i;
    if (!(P->Ei[i] > 0.0)) {
      for (int c = 0; c < 6; ++c) vnew[c] = vn[c];
      continue;
    }
    const double Ki = P->Ei[i] / (3.0 * (1.0 - 2.0 * P->nu)), Gi = P->Ei[i] / (2.0 * (1.0 + P->nu));
    const double tauK = P->taui[i] * P->Ei[i] / Ki, tauG = P->taui[i] * P->Ei[i] / Gi;
    /* V_i = a (3 K_i tauK P1 + 2 G_i tauG P2): F_i = P1 / (3 a K_i tauK) + P2 / (2 a G_i tauG);
       F_i C_i = P1 / (a tauK) + P2 / (a tauG) */
    const ocx lv = 1.0 / (a * tauK), ld = 1.0 / (a * tauG);
    double vnd[6];
    ocx vn_m;
    {
      ocx t6[6], td[6];
      for (int c = 0; c < 6; ++c) t6[c] = vn[c];
      split(t6, &vn_m, td);
      for (int c = 0; c < 6; ++c) vnd[c] = creal(td[c]);
    }
    /* implicit Euler: v^{n+1} = v^n + dt lambda (e* - v^{n+1}) per projector */
    const ocx vm = (vn_m + dt * lv * es_m) / (1.0 + dt * lv);
    ocx vd[6];
    for (int c = 0; c < 6; ++c) vd[c] = (vnd[c] + dt * ld * es_d[c]) / (1.0 + dt * ld);
    ocx sv[6], dv[6];
    for (int c = 0; c < 6; ++c) {
      vnew[c] = vm * M1[c] + vd[c];
      dv[c] = vnew[c] - vn[c];
      sv[c] = 3.0 * Ki * (es_m - vm) * M1[c] + 2.0 * Gi * (es_d[c] - vd[c]); /* sigma_v,i */
      sig[c] += sv[c];
    }
    const ocx trdv = dv[0] + dv[1] + dv[2];
    trdev_sum += 3.0 * Ki * P->alpha * ((treps - treps_n) - trdv);
    for (int c = 0; c < 6; ++c) visc += sv[c] * dv[c];
  }
  ocx sm, sd[6];
  split(sig, &sm, sd);
  ocx s2 = 0.0;
  for (int c = 0; c < 6; ++c) s2 += sd[c] * sd[c];
  *q = csqrt(1.5 * s2);
  const ocx p1 = zn[6] + dp;
  const ocx H = creal(p1) > 0.0 ? G1 * P->k * cpow(p1, P->n) : 0.0;
  const ocx dH_dth = -P->beta1 * H;
  for (int c = 0; c < 6; ++c) { o->sig[c] = sig[c]; o->znew[c] = evp[c]; }
  o->znew[6] = p1;
  (void)G2;
  o->D = (-theta * (3.0 * Kinf * P->alpha * (treps - treps_n) + trdev_sum) + theta * dH_dth * dp +
          sy * dp + visc) / dt;
  o->diss = (sy * dp + visc) / dt;
}

/* residual of the viscoplastic step: g(dp) = dp - dt p_dot(q(dp), p^n + dp) */
static ocx pa66_g(const opa66 *P, const ocx eps[6], ocx theta, const double *zn, double trn,
                  double dt, ocx dp, const ocx ntr[6], opa66_out *o) {
  ocx q;
  pa66_at(P, eps, theta, zn, trn, dt, dp, ntr, &q, o);
  const ocx x = theta - P->theta_ref;
  const ocx G1 = cexp(-P->beta1 * x), G2 = cexp(-P->beta2 * x);
  const ocx sy = G1 * P->sy0, eta = G2 * P->eta0;
  const ocx p1 = zn[6] + dp;
  const ocx H = creal(p1) > 0.0 ? G1 * P->k * cpow(p1, P->n) : 0.0;
  ocx phi = (q - sy - H) / sy;
  if (creal(phi) < 0.0) phi = 0.0;
  return dp - dt * (sy / eta) * cpow(phi, P->m);
}

/* the PA66 law for one complex input: trial at dp = 0, then the return */
static void pa66_eval(const opa66 *P, const ocx eps[6], ocx theta, const double *zn, double trn,
                      double dt, int *plastic_io, opa66_out *o) {
  const ocx zero6[6] = {0, 0, 0, 0, 0, 0};
  ocx q;
  pa66_at(P, eps, theta, zn, trn, dt, 0.0, zero6, &q, o);
  const ocx x = theta - P->theta_ref;
  const ocx G1 = cexp(-P->beta1 * x);
  const ocx sy = G1 * P->sy0;
  const ocx Hn = zn[6] > 0.0 ? G1 * P->k * cpow(zn[6], P->n) : 0.0;
  /* the decision elastic / viscoplastic is taken once, on the real input */
  if (*plastic_io < 0) *plastic_io = creal(q - sy - Hn) > 0.0;
  if (!*plastic_io) return;
  /* unit trial deviator */
  ocx sm, sd[6], ntr[6];
  split(o->sig, &sm, sd);
  ocx s2 = 0.0;
  for (int c = 0; c < 6; ++c) s2 += sd[c] * sd[c];
  const ocx sn = csqrt(s2);
  for (int c = 0; c < 6; ++c) ntr[c] = sd[c] / sn;
  /* bracket and bisect on the real parts: g is increasing in dp */
  double lo = 0.0, hi = 1e-8;
  opa66_out tmp;
  const ocx epsr[6] = {creal(eps[0]), creal(eps[1]), creal(eps[2]), creal(eps[3]), creal(eps[4]),
                       creal(eps[5])};
  const ocx ntrr[6] = {creal(ntr[0]), creal(ntr[1]), creal(ntr[2]), creal(ntr[3]), creal(ntr[4]),
                       creal(ntr[5])};
  const ocx thr = creal(theta);
  for (int it = 0; it < 200 && creal(pa66_g(P, epsr, thr, zn, trn, dt, hi, ntrr, &tmp)) <= 0.0; ++it)
    hi *= 2.0;
  for (int it = 0; it < 300 && hi - lo > 1e-17 * hi; ++it) {
    const double mid = 0.5 * (lo + hi);
    if (creal(pa66_g(P, epsr, thr, zn, trn, dt, mid, ntrr, &tmp)) > 0.0) hi = mid;
    else lo = mid;
  }
  ocx dp = 0.5 * (lo + hi);
  /* Newton steps in complex arithmetic carry d dp / d input (derivative of g
     by a real central difference; the steps converge the imaginary part) */
  const double h = 1e-7 * (creal(dp) > 0.0 ? creal(dp) : 1e-12);
  const double gp = (creal(pa66_g(P, epsr, thr, zn, trn, dt, creal(dp) + h, ntrr, &tmp)) -
                     creal(pa66_g(P, epsr, thr, zn, trn, dt, creal(dp) - h, ntrr, &tmp))) / (2.0 * h);
  for (int it = 0; it < 4; ++it) dp -= pa66_g(P, eps, theta, zn, trn, dt, dp, ntr, o) / gp;
  pa66_g(P, eps, theta, zn, trn, dt, dp, ntr, o);
}

static void pa66_leaf(const double *row, const double eps[6], double theta, const double *zn,
                      double trn, double dt, oleaf *L) {
  opa66 P;
  pa66_params(row, &P);
  const double h = 1e-30;
  opa66_out o;
  ocx e[6];
  for (int c = 0; c < 6; ++c) e[c] = eps[c];
  int plastic = -1;
  pa66_eval(&P, e, theta, zn, trn, dt, &plastic, &o);
  for (int c = 0; c < 6; ++c) L->sig[c] = creal(o.sig[c]);
  L->D = creal(o.D);
  L->diss = creal(o.diss);
  for (int c = 0; c < OR_ZMAX; ++c) L->znew[c] = creal(o.znew[c]);
  /* complex-step derivatives in the six strain directions and in theta */
  for (int j = 0; j < 7; ++j) {
    for (int c = 0; c < 6; ++c) e[c] = eps[c] + (c == j ? I * h : 0.0);
    const ocx th = theta + (j == 6 ? I * h : 0.0);
    opa66_out od;
    pa66_eval(&P, e, th, zn, trn, dt, &plastic, &od);
    for (int c = 0; c < 6; ++c) {
      if (j < 6) L->C[c][j] = cimag(od.sig[c]) / h;
      else L->tau[c] = cimag(od.sig[c]) / h;
    }
    if (j < 6) L->d[j] = cimag(od.D) / h;
    else L->g = cimag(od.D) / h;
  }
}

/* eps: Mandel strain at t^{n+1}; trn: trace of the leaf strain at t^n (kinds 0
   and 1; kind 2 takes its strain at t^n from zn); zn: internal variables of
   the leaf at t^n (kinds 1 and 2) */
void oracle_leaf(const double *matp, const double eps[6], double theta, const double *zn,
                 double trn, double dt, double *outp) {
  if ((int)matp[0] == 3) {
    oleaf L3;
    memset(&L3, 0, sizeof(L3));
    pa66_leaf(matp, eps, theta, zn, trn, dt, &L3);
    double *o = outp;
    memcpy(o, L3.sig, 6 * sizeof(double)); o += 6;
    memcpy(o, L3.C, 36 * sizeof(double)); o += 36;
    memcpy(o, L3.tau, 6 * sizeof(double)); o += 6;
    *o++ = L3.D;
    memcpy(o, L3.d, 6 * sizeof(double)); o += 6;
    *o++ = L3.g;
    *o++ = L3.diss;
    memcpy(o, L3.znew, OR_ZMAX * sizeof(double));
    return;
  }
  omat m;
  m.kind = (int)matp[0];
  m.E = matp[1]; m.nu = matp[2]; m.alpha = matp[3]; m.theta0 = matp[4];
  m.sy0 = matp[5]; m.dsy_dT = matp[6]; m.H = matp[7];
  m.m_rate = matp[8]; m.t_visc = matp[9]; m.dE_dT = matp[10];
  oleaf L;
  memset(&L, 0, sizeof(L));
  /* moduli: E(theta) = E r(theta), r = 1 + dE_dT (theta - theta0) for kind 2
     (floored at 1e-3), r = 1 otherwise */
  double r = 1.0, dr = 0.0;
  if (m.kind == 2) {
    r = 1.0 + m.dE_dT * (theta - m.theta0);
    dr = m.dE_dT;
    if (r < 1e-3) { r = 1e-3; dr = 0.0; }
  }
  const double Kb = r * m.E / (3.0 * (1.0 - 2.0 * m.nu));
  const double G = r * m.E / (2.0 * (1.0 + m.nu));
  const double dKb = dr * m.E / (3.0 * (1.0 - 2.0 * m.nu)); /* dK/dtheta */
  const double dG = dr * m.E / (2.0 * (1.0 + m.nu));        /* dG/dtheta */
  double ee[6];
  for (int c = 0; c < 6; ++c) ee[c] = eps[c] - M1[c] * m.alpha * (theta - m.theta0);
  if (m.kind >= 1)
    for (int c = 0; c < 6; ++c) ee[c] -= zn[c];
  double tr = ee[0] + ee[1] + ee[2];
  double dev[6];
  for (int c = 0; c < 6; ++c) dev[c] = ee[c] - M1[c] * tr / 3.0;
  /* elastic predictor sigma = K tr(ee) I + 2G dev(ee) */
  for (int c = 0; c < 6; ++c) L.sig[c] = Kb * tr * M1[c] + 2.0 * G * dev[c];
  /* C = 3K P1 + 2G P2, P1 = m m^T / 3, P2 = I - P1 */
  for (int a = 0; a < 6; ++a)
    for (int b = 0; b < 6; ++b) {
      double p1 = M1[a] * M1[b] / 3.0;
      double p2 = (a == b ? 1.0 : 0.0) - p1;
      L.C[a][b] = 3.0 * Kb * p1 + 2.0 * G * p2;
    }
  /* dsigma/dtheta at fixed strain and internal variables */
  for (int c = 0; c < 6; ++c)
    L.tau[c] = -3.0 * Kb * m.alpha * M1[c] + dKb * tr * M1[c] + 2.0 * dG * dev[c];
  /* strain increment of the step (its trace for kinds 0 and 1) */
  double de[6] = {0, 0, 0, 0, 0, 0}, trde;
  if (m.kind == 2) {
    for (int c = 0; c < 6; ++c) de[c] = eps[c] - zn[7 + c];
    trde = de[0] + de[1] + de[2];
  } else {
    trde = (eps[0] + eps[1] + eps[2]) - trn;
  }
  L.D = -3.0 * Kb * m.alpha * theta * trde / dt;
  for (int c = 0; c < 6; ++c) L.d[c] = -3.0 * Kb * m.alpha * theta * M1[c] / dt;
  L.g = -3.0 * m.alpha * (Kb + dKb * theta) * trde / dt;
  L.diss = 0.0;
  if (m.kind >= 1) {
    for (int c = 0; c < 7; ++c) L.znew[c] = zn[c];
    if (m.kind == 2)
      for (int c = 0; c < 6; ++c) L.znew[7 + c] = eps[c];
    double sy = m.sy0 + m.dsy_dT * (theta - m.theta0);
    double dsy = m.dsy_dT;
    if (sy < 1e-6) { sy = 1e-6; dsy = 0.0; }
    double s[6], snorm2 = 0.0;
    for (int c = 0; c < 6; ++c) { s[c] = 2.0 * G * dev[c]; snorm2 += s[c] * s[c]; }
    double snorm = sqrt(snorm2);
    double qtr = sqrt(1.5) * snorm;
    double f = qtr - sy - m.H * zn[6];
    double dp = 0.0, q = qtr, kk = 0.0, ddp_dth = 0.0, N[6] = {0, 0, 0, 0, 0, 0};
    if (f > 0.0) {
      double kinv, phi = 0.0; /* kinv = d dp / d q_trial */
      if (m.kind == 1) {
        dp = f / (3.0 * G + m.H);
        kinv = 1.0 / (3.0 * G + m.H);
      } else {
        /* implicit Euler of the Perzyna law: Newton on
           g(x) = x - c phi(x)^m, phi(x) = (f - (3G + H) x) / sigma_Y, which is
           increasing and concave on [0, f / (3G + H)], so Newton from x = 0
           increases monotonically to the root */
        const double c = dt / m.t_visc, me = m.m_rate, xmax = f / (3.0 * G + m.H);
        double x = 0.0;
        for (int it = 0; it < 200; ++it) {
          phi = (f - (3.0 * G + m.H) * x) / sy;
          if (phi < 0.0) phi = 0.0;
          const double gx = x - c * pow(phi, me);
          const double gp = 1.0 + c * me * pow(phi, me - 1.0) * (3.0 * G + m.H) / sy;
          double xn = x - gx / gp;
          if (xn < 0.0) xn = 0.0;
          if (xn > xmax) xn = xmax;
          const double step = fabs(xn - x);
          x = xn;
          if (step <= 1e-16 * x) break;
        }
        dp = x;
        phi = (f - (3.0 * G + m.H) * dp) / sy;
        if (phi < 0.0) phi = 0.0;
        const double cm = c * me * pow(phi, me - 1.0);
        kinv = cm / (sy + cm * (3.0 * G + m.H)); /* 1 / (3G + H + h_v) */
      }
      for (int c = 0; c < 6; ++c) N[c] = s[c] / snorm;
      for (int c = 0; c < 6; ++c) {
        L.sig[c] -= 2.0 * G * sqrt(1.5) * dp * N[c];
        L.znew[c] = zn[c] + sqrt(1.5) * dp * N[c];
      }
      L.znew[6] = zn[6] + dp;
      q = qtr - 3.0 * G * dp;
      double th1 = 1.0 - 3.0 * G * dp / qtr;
      double thb = 3.0 * G * kinv - 3.0 * G * dp / qtr;
      for (int a = 0; a < 6; ++a)
        for (int b = 0; b < 6; ++b) {
          double p1 = M1[a] * M1[b] / 3.0;
          double p2 = (a == b ? 1.0 : 0.0) - p1;
          L.C[a][b] = 3.0 * Kb * p1 + 2.0 * G * th1 * p2 - 2.0 * G * thb * N[a] * N[b];
        }
      /* d dp / d theta from the flow equation at fixed strain */
      const double dqtr = G > 0.0 ? (dG / G) * qtr : 0.0;
      ddp_dth = (dqtr - 3.0 * dG * dp - dsy - phi * dsy) * kinv;
      const double dq = dqtr - 3.0 * dG * dp - 3.0 * G * ddp_dth;
      /* deviatoric part of dsigma/dtheta: sqrt(2/3) dq/dtheta N */
      for (int c = 0; c < 6; ++c) L.tau[c] += sqrt(2.0 / 3.0) * (dq - dqtr) * N[c];
      kk = sqrt(1.5) * 2.0 * G * kinv; /* d dp / d eps = kk N */
      L.D += sy * dp / dt;
      L.diss = sy * dp / dt;
      for (int c = 0; c < 6; ++c) L.d[c] += sy * kk * N[c] / dt;
      L.g += (dsy * dp + sy * ddp_dth) / dt;
    }
    if (m.kind == 2) {
      /* theta (r'/r) sigma : (de - deps_p) and its derivatives */
      const double sf = dr / r, dsf = -sf * sf;
      double v[6], sv = 0.0, tv = 0.0, Cv[6];
      for (int c = 0; c < 6; ++c) {
        v[c] = de[c] - sqrt(1.5) * dp * N[c];
        sv += L.sig[c] * v[c];
        tv += L.tau[c] * v[c];
      }
      for (int a = 0; a < 6; ++a) {
        Cv[a] = 0.0;
        for (int b = 0; b < 6; ++b) Cv[a] += L.C[a][b] * v[b];
      }
      L.D += theta * sf * sv / dt;
      for (int c = 0; c < 6; ++c) L.d[c] += theta * sf * (Cv[c] + L.sig[c] - q * kk * N[c]) / dt;
      L.g += ((sf + theta * dsf) * sv + theta * sf * (tv - q * ddp_dth)) / dt;
    }
  }
  /* pack: sig 6, C 36, tau 6, D, d 6, g, diss, znew 79 = 136 */
  double *o = outp;
  memcpy(o, L.sig, 6 * sizeof(double)); o += 6;
  memcpy(o, L.C, 36 * sizeof(double)); o += 36;
  memcpy(o, L.tau, 6 * sizeof(double)); o += 6;
  *o++ = L.D;
  memcpy(o, L.d, 6 * sizeof(double)); o += 6;
  *o++ = L.g;
  *o++ = L.diss;
  memcpy(o, L.znew, OR_ZMAX * sizeof(double));
}

static void leaf_eval(const omat *m, const double eps[6], double theta, const double *zn,
                      double trn, double dt, oleaf *L) {
  double o[57 + OR_ZMAX];
  oracle_leaf(m->row, eps, theta, zn, trn, dt, o);
  memcpy(L->sig, o, 6 * sizeof(double));
  memcpy(L->C, o + 6, 36 * sizeof(double));
  memcpy(L->tau, o + 42, 6 * sizeof(double));
  L->D = o[48];
  memcpy(L->d, o + 49, 6 * sizeof(double));
  L->g = o[55];
  L->diss = o[56];
  memcpy(L->znew, o + 57, OR_ZMAX * sizeof(double));
}

/* ------------------------------------------------------------------ */
/* one Gauss point                                                      */
/* ------------------------------------------------------------------ */

typedef struct {
  double tol, gamma, res_floor;
  int maxit, maxbacktrack, dense;
} oopts;

typedef struct {
  const otree *t;
  const omat *mats;
  const oopts *o;
  double eps_bar[6], theta, dt;
  const double *zn;        /* state_in (for z offsets) */
  double trn[1 << OR_MAXK];
  oleaf *leaf;             /* [nleaf] */
  double *a;               /* [3 nnode] */
  double sig_bar[6];
  double res;
} opoint;

/* leaf strains from explicit A:  eps_j = eps_bar + sum_k s_{p,j} B_p a_p */
static void leaf_strain(const otree *t, const double *eps_bar, const double *a, int j,
                        double eps[6]) {
  for (int c = 0; c < 6; ++c) eps[c] = eps_bar[c];
  for (int k = 0; k < t->K; ++k) {
    int p = t->anc[j][k];
    double B[6][3];
    bmat(t->n[p], B);
    for (int c = 0; c < 6; ++c)
      eps[c] += t->s[j][k] * (B[c][0] * a[3 * p] + B[c][1] * a[3 * p + 1] + B[c][2] * a[3 * p + 2]);
  }
}

/* Residual function of Algorithm 1 (also stores leaf results) */
static double residual(opoint *P) {
  const otree *t = P->t;
  double r[3 * (1 << OR_MAXK)];
  memset(r, 0, sizeof(double) * 3 * t->nnode);
  for (int c = 0; c < 6; ++c) P->sig_bar[c] = 0.0;
  for (int j = 0; j < t->nleaf; ++j) {
    double eps[6];
    leaf_strain(t, P->eps_bar, P->a, j, eps);
    const double *zj = t->zoff[j] >= 0 ? P->zn + t->zoff[j] : NULL;
    leaf_eval(&P->mats[t->phase[j]], eps, P->theta, zj, P->trn[j], P->dt, &P->leaf[j]);
    for (int c = 0; c < 6; ++c) P->sig_bar[c] += t->w[j] * P->leaf[j].sig[c];
    /* r = A^T W sigma */
    for (int k = 0; k < t->K; ++k) {
      int p = t->anc[j][k];
      double B[6][3];
      bmat(t->n[p], B);
      for (int e = 0; e < 3; ++e) {
        double acc = 0.0;
        for (int c = 0; c < 6; ++c) acc += B[c][e] * P->leaf[j].sig[c];
        r[3 * p + e] += t->w[j] * t->s[j][k] * acc;
      }
    }
  }
  double rn = 0.0, sn = 0.0;
  for (int e = 0; e < 3 * t->nnode; ++e) rn += r[e] * r[e];
  for (int c = 0; c < 6; ++c) sn += P->sig_bar[c] * P->sig_bar[c];
  double den = sqrt(sn);
  if (den < P->o->res_floor) den = P->o->res_floor;
  return sqrt(rn) / ((double)t->nnode * den);
}

/* ---- sparse (ancestor-structured) block Cholesky -------------------- */
/* S[p][d] holds block (row q, col p) for q = ancestor of p at level d+1,
   d = 0..depth(p)-1 (q = p when d = depth(p)-1).                         */
typedef struct {
  int nnode, K;
  double *S; /* [nnode][K][3][3] */
} osparse;

#define SBLK(M, p, d) ((M)->S + ((size_t)(p) * (M)->K + (d)) * 9)

/* node q's ancestor at level k (k <= depth(q)): via any leaf under q */
static int ancestor_at(const otree *t, int q, int k) {
  /* node q = (kq, iq); ancestor at level k has position ((iq-1) >> (kq-k)) + 1 */
  int kq = t->depth[q];
  int iq = q - ((1 << t->K) - (1 << kq)) + 1;
  int i = ((iq - 1) >> (kq - k)) + 1;
  return pidx(t->K, k, i);
}

static void assemble_sparse(const opoint *P, osparse *M) {
  const otree *t = P->t;
  memset(M->S, 0, sizeof(double) * (size_t)t->nnode * t->K * 9);
  for (int j = 0; j < t->nleaf; ++j) {
    const oleaf *L = &P->leaf[j];
    double CB[OR_MAXK][6][3];
    double Bs[OR_MAXK][6][3];
    for (int k = 0; k < t->K; ++k) {
      bmat(t->n[t->anc[j][k]], Bs[k]);
      for (int a = 0; a < 6; ++a)
        for (int e = 0; e < 3; ++e) {
          double acc = 0.0;
          for (int b = 0; b < 6; ++b) acc += L->C[a][b] * Bs[k][b][e];
          CB[k][a][e] = acc;
        }
    }
    /* block (row q at level kq, col p at level kp), kq <= kp */
    for (int kp = 0; kp < t->K; ++kp)
      for (int kq = 0; kq <= kp; ++kq) {
        int p = t->anc[j][kp];
        double f = t->w[j] * t->s[j][kp] * t->s[j][kq];
        double *blk = SBLK(M, p, kq);
        for (int e = 0; e < 3; ++e)
          for (int h = 0; h < 3; ++h) {
            double acc = 0.0;
            for (int a = 0; a < 6; ++a) acc += Bs[kq][a][e] * CB[kp][a][h];
            blk[3 * e + h] += f * acc;
          }
      }
  }
}

static int chol3(const double A[9], double L[9]) {
  memset(L, 0, 9 * sizeof(double));
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j <= i; ++j) {
      double s = A[3 * i + j];
      for (int k = 0; k < j; ++k) s -= L[3 * i + k] * L[3 * j + k];
      if (i == j) {
        if (!(s > 0.0)) return -1;
        L[3 * i + i] = sqrt(s);
      } else {
        L[3 * i + j] = s / L[3 * j + j];
      }
    }
  return 0;
}

/* factor in paper order (descendants first); L overwrites S */
static int factor_sparse(const otree *t, osparse *M) {
  for (int p = 0; p < t->nnode; ++p) {
    int kp = t->depth[p];
    double Lpp[9];
    if (chol3(SBLK(M, p, kp - 1), Lpp)) return -1;
    memcpy(SBLK(M, p, kp - 1), Lpp, sizeof(Lpp));
    /* L_qp = H_qp L_pp^{-T} for every ancestor q */
    for (int d = 0; d < kp - 1; ++d) {
      double *H = SBLK(M, p, d);
      double X[9];
      for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) {
          double s = H[3 * r + c];
          for (int k = 0; k < c; ++k) s -= X[3 * r + k] * Lpp[3 * c + k];
          X[3 * r + c] = s / Lpp[3 * c + c];
        }
      memcpy(H, X, sizeof(X));
    }
    /* H_{q1 q2} -= L_{q1 p} L_{q2 p}^T, q1 at level d1 <= d2 (q1 ancestor of q2) */
    for (int d2 = 0; d2 < kp - 1; ++d2) {
      int q2 = ancestor_at(t, p, d2 + 1);
      for (int d1 = 0; d1 <= d2; ++d1) {
        const double *L1 = SBLK(M, p, d1), *L2 = SBLK(M, p, d2);
        double *T = SBLK(M, q2, d1);
        for (int r = 0; r < 3; ++r)
          for (int c = 0; c < 3; ++c) {
            double s = 0.0;
            for (int k = 0; k < 3; ++k) s += L1[3 * r + k] * L2[3 * c + k];
            T[3 * r + c] -= s;
          }
      }
    }
  }
  return 0;
}

/* solve L L^T x = b in place */
static void solve_sparse(const otree *t, const osparse *M, double *b) {
  for (int p = 0; p < t->nnode; ++p) {
    int kp = t->depth[p];
    const double *Lpp = SBLK(M, p, kp - 1);
    double y[3];
    for (int r = 0; r < 3; ++r) {
      double s = b[3 * p + r];
      for (int k = 0; k < r; ++k) s -= Lpp[3 * r + k] * y[k];
      y[r] = s / Lpp[3 * r + r];
    }
    for (int r = 0; r < 3; ++r) b[3 * p + r] = y[r];
    for (int d = 0; d < kp - 1; ++d) {
      int q = ancestor_at(t, p, d + 1);
      const double *Lq = SBLK(M, p, d);
      for (int r = 0; r < 3; ++r)
        b[3 * q + r] -= Lq[3 * r] * y[0] + Lq[3 * r + 1] * y[1] + Lq[3 * r + 2] * y[2];
    }
  }
  for (int p = t->nnode - 1; p >= 0; --p) {
    int kp = t->depth[p];
    double z[3] = {b[3 * p], b[3 * p + 1], b[3 * p + 2]};
    for (int d = 0; d < kp - 1; ++d) {
      int q = ancestor_at(t, p, d + 1);
      const double *Lq = SBLK(M, p, d);
      for (int c = 0; c < 3; ++c)
        z[c] -= Lq[c] * b[3 * q] + Lq[3 + c] * b[3 * q + 1] + Lq[6 + c] * b[3 * q + 2];
    }
    const double *Lpp = SBLK(M, p, kp - 1);
    for (int r = 2; r >= 0; --r) {
      double s = z[r];
      for (int k = r + 1; k < 3; ++k) s -= Lpp[3 * k + r] * b[3 * p + k];
      b[3 * p + r] = s / Lpp[3 * r + r];
    }
  }
}

/* ---- dense path: dense A, dense Hessian, dense Cholesky -------------- */
typedef struct {
  int nr, nc;     /* 6 nleaf x 3 nnode */
  double *A;      /* row-major */
  double *H;      /* nc x nc */
} odense;

static void build_dense_A(const otree *t, odense *D) {
  D->nr = 6 * t->nleaf;
  D->nc = 3 * t->nnode;
  memset(D->A, 0, sizeof(double) * D->nr * D->nc);
  for (int j = 0; j < t->nleaf; ++j)
    for (int k = 0; k < t->K; ++k) {
      int p = t->anc[j][k];
      double B[6][3];
      bmat(t->n[p], B);
      for (int c = 0; c < 6; ++c)
        for (int e = 0; e < 3; ++e) D->A[(size_t)(6 * j + c) * D->nc + 3 * p + e] = t->s[j][k] * B[c][e];
    }
}

static void assemble_dense(const opoint *P, odense *D) {
  const otree *t = P->t;
  int nc = D->nc;
  /* WCA = W blockdiag(C) A  (6 nleaf x nc) */
  double *WCA = (double *)calloc((size_t)D->nr * nc, sizeof(double));
  for (int j = 0; j < t->nleaf; ++j)
    for (int a = 0; a < 6; ++a)
      for (int col = 0; col < nc; ++col) {
        double s = 0.0;
        for (int b = 0; b < 6; ++b) s += P->leaf[j].C[a][b] * D->A[(size_t)(6 * j + b) * nc + col];
        WCA[(size_t)(6 * j + a) * nc + col] = t->w[j] * s;
      }
  for (int r = 0; r < nc; ++r)
    for (int c = 0; c < nc; ++c) {
      double s = 0.0;
      for (int i = 0; i < D->nr; ++i) s += D->A[(size_t)i * nc + r] * WCA[(size_t)i * nc + c];
      D->H[(size_t)r * nc + c] = s;
    }
  free(WCA);
}

static int factor_dense(odense *D) {
  int n = D->nc;
  double *H = D->H;
  for (int j = 0; j < n; ++j) {
    double s = H[(size_t)j * n + j];
    for (int k = 0; k < j; ++k) s -= H[(size_t)j * n + k] * H[(size_t)j * n + k];
    if (!(s > 0.0)) return -1;
    double d = sqrt(s);
    H[(size_t)j * n + j] = d;
    for (int i = j + 1; i < n; ++i) {
      double v = H[(size_t)i * n + j];
      for (int k = 0; k < j; ++k) v -= H[(size_t)i * n + k] * H[(size_t)j * n + k];
      H[(size_t)i * n + j] = v / d;
    }
  }
  return 0;
}

static void solve_dense(const odense *D, double *b) {
  int n = D->nc;
  const double *L = D->H;
  for (int i = 0; i < n; ++i) {
    double s = b[i];
    for (int k = 0; k < i; ++k) s -= L[(size_t)i * n + k] * b[k];
    b[i] = s / L[(size_t)i * n + i];
  }
  for (int i = n - 1; i >= 0; --i) {
    double s = b[i];
    for (int k = i + 1; k < n; ++k) s -= L[(size_t)k * n + i] * b[k];
    b[i] = s / L[(size_t)i * n + i];
  }
}

/* ---- linear algebra front-end shared by the Newton step and tangents */
typedef struct {
  osparse sp;
  odense dn;
  int dense;
} osolver;

static int factor(const opoint *P, osolver *S) {
  if (S->dense) {
    assemble_dense(P, &S->dn);
    return factor_dense(&S->dn);
  }
  assemble_sparse(P, &S->sp);
  return factor_sparse(P->t, &S->sp);
}

static void solve(const opoint *P, const osolver *S, double *b) {
  if (S->dense) solve_dense(&S->dn, b);
  else solve_sparse(P->t, &S->sp, b);
}

/* b = -A^T W v, with v_j a 6-vector per leaf (given as callback data) */
static void rhs_from_leaf_vectors(const otree *t, const double *v /* [nleaf][6] */, double *b) {
  memset(b, 0, sizeof(double) * 3 * t->nnode);
  for (int j = 0; j < t->nleaf; ++j)
    for (int k = 0; k < t->K; ++k) {
      int p = t->anc[j][k];
      double B[6][3];
      bmat(t->n[p], B);
      for (int e = 0; e < 3; ++e) {
        double acc = 0.0;
        for (int c = 0; c < 6; ++c) acc += B[c][e] * v[6 * j + c];
        b[3 * p + e] -= t->w[j] * t->s[j][k] * acc;
      }
    }
}

/* A_j x  for leaf j (6-vector) */
static void apply_A_leaf(const otree *t, int j, const double *x, double out[6]) {
  for (int c = 0; c < 6; ++c) out[c] = 0.0;
  for (int k = 0; k < t->K; ++k) {
    int p = t->anc[j][k];
    double B[6][3];
    bmat(t->n[p], B);
    for (int c = 0; c < 6; ++c)
      out[c] += t->s[j][k] * (B[c][0] * x[3 * p] + B[c][1] * x[3 * p + 1] + B[c][2] * x[3 * p + 2]);
  }
}

enum { OPT_OK = 0, OPT_NOT_CONVERGED = 1, OPT_NONFINITE = 2 };

/* Algorithm 1 for one Gauss point.  res_hist (optional) receives the
   residual after the warm start and after every Newton iteration. */
static int eval_point(const otree *t, const omat *mats, const oopts *o, const double deps[6],
                      double theta, double dt, const double *sin, double *sout, double *out,
                      int *iters_out, double *res_hist, int nhist) {
  int nn = t->nnode;
  opoint P;
  memset(&P, 0, sizeof(P));
  P.t = t;
  P.mats = mats;
  P.o = o;
  P.theta = theta;
  P.dt = dt;
  P.zn = sin;
  for (int c = 0; c < 6; ++c) P.eps_bar[c] = sin[c] + deps[c];
  P.leaf = (oleaf *)calloc(t->nleaf, sizeof(oleaf));
  P.a = (double *)calloc(3 * nn, sizeof(double));
  double *da = (double *)calloc(3 * nn, sizeof(double));
  osolver S;
  memset(&S, 0, sizeof(S));
  S.dense = o->dense;
  if (S.dense) {
    S.dn.A = (double *)calloc((size_t)6 * t->nleaf * 3 * nn, sizeof(double));
    S.dn.H = (double *)calloc((size_t)9 * nn * nn, sizeof(double));
    build_dense_A(t, &S.dn);
  } else {
    S.sp.nnode = nn;
    S.sp.K = t->K;
    S.sp.S = (double *)calloc((size_t)nn * t->K * 9, sizeof(double));
  }
  /* previous leaf strain traces from eps_bar^n and a^n */
  for (int j = 0; j < t->nleaf; ++j) {
    double en[6];
    leaf_strain(t, sin, sin + 8, j, en);
    P.trn[j] = en[0] + en[1] + en[2];
  }
  /* warm start: a^{n+1} <- a^n */
  for (int e = 0; e < 3 * nn; ++e) P.a[e] = sin[8 + e];
  double res = residual(&P);
  int h = 0;
  if (res_hist && h < nhist) res_hist[h++] = res;
  int it = 0, status = OPT_NOT_CONVERGED;
  int fact_fail = 0;
  for (it = 1; it <= o->maxit; ++it) {
    if (!isfinite(res)) break;
    /* solve [A^T W dsigma/deps A] da = -A^T W sigma */
    if (factor(&P, &S)) { fact_fail = 1; break; }
    double *sig = (double *)malloc(sizeof(double) * 6 * t->nleaf);
    for (int j = 0; j < t->nleaf; ++j)
      for (int c = 0; c < 6; ++c) sig[6 * j + c] = P.leaf[j].sig[c];
    rhs_from_leaf_vectors(t, sig, da);
    free(sig);
    solve(&P, &S, da);
    /* Backtracking */
    double res_old = res;
    for (int e = 0; e < 3 * nn; ++e) P.a[e] += da[e];
    res = residual(&P);
    double gi = 1.0;
    for (int i = 0; i < o->maxbacktrack; ++i) {
      if (res < res_old) break;
      for (int e = 0; e < 3 * nn; ++e) P.a[e] -= gi * (1.0 - o->gamma) * da[e];
      res = residual(&P);
      gi *= o->gamma;
    }
    if (res_hist && h < nhist) res_hist[h++] = res;
    if (res < o->tol) { status = OPT_OK; break; }
  }
  if (it > o->maxit) it = o->maxit;
  if (!isfinite(res) || fact_fail) status = OPT_NONFINITE;
  if (iters_out) *iters_out = it;

  /* post-convergence: state update and outputs (leaf data of the last
     Residual call are at the final a) */
  double *o_sig = out, *o_C = out + 6, *o_Ct = out + 42, *o_D = out + 48, *o_De = out + 49,
         *o_Dt = out + 55, *o_Diss = out + 56;
  for (int c = 0; c < 57; ++c) out[c] = 0.0;
  int ok_fact = (factor(&P, &S) == 0);
  if (ok_fact) {
    /* seven right-hand sides: da/deps_bar (6 columns) and da/dtheta */
    double *X = (double *)calloc((size_t)7 * 3 * nn, sizeof(double));
    double *v = (double *)malloc(sizeof(double) * 6 * t->nleaf);
    for (int m = 0; m < 6; ++m) {
      for (int j = 0; j < t->nleaf; ++j)
        for (int c = 0; c < 6; ++c) v[6 * j + c] = P.leaf[j].C[c][m];
      rhs_from_leaf_vectors(t, v, X + (size_t)m * 3 * nn);
      solve(&P, &S, X + (size_t)m * 3 * nn);
    }
    for (int j = 0; j < t->nleaf; ++j)
      for (int c = 0; c < 6; ++c) v[6 * j + c] = P.leaf[j].tau[c];
    rhs_from_leaf_vectors(t, v, X + (size_t)6 * 3 * nn);
    solve(&P, &S, X + (size_t)6 * 3 * nn);
    free(v);
    for (int j = 0; j < t->nleaf; ++j) {
      const oleaf *L = &P.leaf[j];
      double wj = t->w[j];
      double Ae[6][6], At[6];
      for (int m = 0; m < 6; ++m) {
        double col[6];
        apply_A_leaf(t, j, X + (size_t)m * 3 * nn, col);
        for (int c = 0; c < 6; ++c) Ae[c][m] = col[c];
      }
      apply_A_leaf(t, j, X + (size_t)6 * 3 * nn, At);
      for (int c = 0; c < 6; ++c) o_sig[c] += wj * L->sig[c];
      /* eq. (ddsdde): C_bar = sum w_j [C_j + C_j A_j da/deps] */
      for (int a = 0; a < 6; ++a)
        for (int m = 0; m < 6; ++m) {
          double s = L->C[a][m];
          for (int b = 0; b < 6; ++b) s += L->C[a][b] * Ae[b][m];
          o_C[6 * a + m] += wj * s;
        }
      /* eq. (ddsddt) */
      for (int a = 0; a < 6; ++a) {
        double s = L->tau[a];
        for (int b = 0; b < 6; ++b) s += L->C[a][b] * At[b];
        o_Ct[a] += wj * s;
      }
      /* eq. (effective coupling term), (drplde), (drpldt), (dissipation) */
      *o_D += wj * L->D;
      for (int m = 0; m < 6; ++m) {
        double s = L->d[m];
        for (int b = 0; b < 6; ++b) s += L->d[b] * Ae[b][m];
        o_De[m] += wj * s;
      }
      {
        double s = L->g;
        for (int b = 0; b < 6; ++b) s += L->d[b] * At[b];
        *o_Dt += wj * s;
      }
      *o_Diss += wj * L->diss;
    }
    free(X);
  } else {
    status = OPT_NONFINITE;
  }
  /* state out */
  memset(sout, 0, sizeof(double) * t->state_words);
  for (int c = 0; c < 6; ++c) sout[c] = P.eps_bar[c];
  sout[6] = theta;
  for (int e = 0; e < 3 * nn; ++e) sout[8 + e] = P.a[e];
  for (int j = 0; j < t->nleaf; ++j)
    if (t->zoff[j] >= 0)
      for (int c = 0; c < z_words(mats[t->phase[j]].kind); ++c) sout[t->zoff[j] + c] = P.leaf[j].znew[c];
  for (int c = 0; c < 57; ++c)
    if (!isfinite(out[c])) status = OPT_NONFINITE;

  free(P.leaf);
  free(P.a);
  free(da);
  if (S.dense) { free(S.dn.A); free(S.dn.H); }
  else free(S.sp.S);
  return status;
}

/* ------------------------------------------------------------------ */
/* exported API (ctypes)                                                */
/* ------------------------------------------------------------------ */

static int load_mats(const double *mats, int n_mats, omat *m) {
  for (int i = 0; i < n_mats; ++i) {
    const double *r = mats + OR_MATW * i;
    m[i].kind = (int)r[0];
    m[i].E = r[1]; m[i].nu = r[2]; m[i].alpha = r[3]; m[i].theta0 = r[4];
    m[i].sy0 = r[5]; m[i].dsy_dT = r[6]; m[i].H = r[7];
    m[i].m_rate = r[8]; m[i].t_visc = r[9]; m[i].dE_dT = r[10];
    memcpy(m[i].row, r, OR_MATW * sizeof(double));
    if (m[i].kind < 0 || m[i].kind > 3) return -1;
    if (m[i].kind == 2 && !(m[i].m_rate >= 1.0 && m[i].t_visc > 0.0)) return -1;
    if (m[i].kind == 3 && !(r[8] >= 1.0 && r[9] > 0.0 && r[5] > 0.0)) return -1;
  }
  return 0;
}

int64_t oracle_state_words(int K, const double *leaf_w, const double *normals, const uint8_t *phase,
                           const double *mats, int n_mats) {
  omat m[256];
  if (n_mats < 1 || n_mats > 256 || load_mats(mats, n_mats, m)) return -1;
  otree *t = (otree *)malloc(sizeof(otree));
  int rc = build_tree(t, K, leaf_w, normals, phase, m, n_mats);
  int64_t w = rc ? rc : t->state_words;
  free(t);
  return w;
}

typedef struct {
  const otree *t;
  const omat *m;
  const oopts *o;
  int64_t n, next;
  pthread_mutex_t lock;
  const double *deps, *theta;
  double dt;
  const double *sin;
  double *sout, *out;
  int32_t *status, *iters;
} ojob;

static void *worker(void *arg) {
  ojob *J = (ojob *)arg;
  for (;;) {
    pthread_mutex_lock(&J->lock);
    int64_t i = J->next++;
    pthread_mutex_unlock(&J->lock);
    if (i >= J->n) break;
    int sw = J->t->state_words;
    int it = 0;
    int st = eval_point(J->t, J->m, J->o, J->deps + 6 * i, J->theta[i], J->dt, J->sin + (size_t)sw * i,
                        J->sout + (size_t)sw * i, J->out + 57 * i, &it, NULL, 0);
    J->status[i] = st;
    J->iters[i] = it;
  }
  return NULL;
}

int oracle_eval_batch(int K, const double *leaf_w, const double *normals, const uint8_t *phase,
                      const double *mats, int n_mats, double tol, int maxit, int maxbacktrack,
                      double gamma, double res_floor, int dense, int64_t n, const double *deps,
                      const double *theta, double dt, const double *state_in, double *state_out,
                      double *out, int32_t *status, int32_t *iters, int nthreads) {
  omat m[256];
  if (n_mats < 1 || n_mats > 256 || load_mats(mats, n_mats, m)) return -1;
  otree *t = (otree *)malloc(sizeof(otree));
  int rc = build_tree(t, K, leaf_w, normals, phase, m, n_mats);
  if (rc) { free(t); return rc; }
  if (dense && K > 7) { free(t); return -6; }
  oopts o = {tol, gamma, res_floor, maxit, maxbacktrack, dense};
  ojob J;
  J.t = t; J.m = m; J.o = &o; J.n = n; J.next = 0;
  pthread_mutex_init(&J.lock, NULL);
  J.deps = deps; J.theta = theta; J.dt = dt; J.sin = state_in; J.sout = state_out; J.out = out;
  J.status = status; J.iters = iters;
  if (nthreads < 1) nthreads = 1;
  if (nthreads > 512) nthreads = 512;
  pthread_t th[512];
  for (int i = 0; i < nthreads; ++i) pthread_create(&th[i], NULL, worker, &J);
  for (int i = 0; i < nthreads; ++i) pthread_join(th[i], NULL);
  pthread_mutex_destroy(&J.lock);
  free(t);
  return 0;
}

/* single point with the residual history of Algorithm 1 */
int oracle_eval_point_trace(int K, const double *leaf_w, const double *normals, const uint8_t *phase,
                            const double *mats, int n_mats, double tol, int maxit, int maxbacktrack,
                            double gamma, double res_floor, int dense, const double *deps, double theta,
                            double dt, const double *state_in, double *state_out, double *out,
                            int32_t *status, int32_t *iters, double *res_hist, int nhist) {
  omat m[256];
  if (n_mats < 1 || n_mats > 256 || load_mats(mats, n_mats, m)) return -1;
  otree *t = (otree *)malloc(sizeof(otree));
  int rc = build_tree(t, K, leaf_w, normals, phase, m, n_mats);
  if (rc) { free(t); return rc; }
  oopts o = {tol, gamma, res_floor, maxit, maxbacktrack, dense};
  int it = 0;
  *status = eval_point(t, m, &o, deps, theta, dt, state_in, state_out, out, &it, res_hist, nhist);
  *iters = it;
  free(t);
  return 0;
}

/* leaf strains eps = eps_bar + A a for all leaves (for kinematic checks) */
int oracle_leaf_strains(int K, const double *leaf_w, const double *normals, const double *eps_bar,
                        const double *a, double *eps_out) {
  omat m[1] = {{0, 1.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0}};
  uint8_t ph[1 << OR_MAXK];
  memset(ph, 0, sizeof(ph));
  otree *t = (otree *)malloc(sizeof(otree));
  int rc = build_tree(t, K, leaf_w, normals, ph, m, 1);
  if (rc) { free(t); return rc; }
  for (int j = 0; j < t->nleaf; ++j) leaf_strain(t, eps_bar, a, j, eps_out + 6 * j);
  free(t);
  return 0;
}
