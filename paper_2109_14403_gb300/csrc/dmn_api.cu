// dmn_api.cu -- the C ABI declared in include/dmn.h: handle creation (tree
// setup of arXiv 2109.14403 Sec. 3.1), state initialisation and the batched
// evaluation launch (Sec. 3.3, Algorithm 1).
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <vector>

#include "../../include/dmn.h"
#include "../../include/dmn_mlp.h"
#include "dmn_internal.h"

using namespace dmn;

struct dmn_handle_s {
  int K, N, nleaf, SW, zend, n_mats;
  dmn_options opt;
  int device, num_sms;
  int blocks_per_sm;     // resident CTAs per SM of the selected kernel variant
  unsigned long long *d_queue;  // work-queue counter (one per handle)
  unsigned long long *d_open;   // dmn_eval_mixed: points still iterating
  double *d_node;        // [N][kNodeWords]
  float *d_node_df;      // [N][kNodeDfl]
  double *d_leafw;       // [nleaf]
  int zw;                // words of internal variables per state block (law 3: words
                         // of the leaves' history in the solve's shared memory)
  int law;               // largest material kind (1: kinds 0/1, 2: Perzyna leaves)
  uint8_t *d_phase;      // [nleaf]
  int *d_zoff;           // [nleaf]
  int *d_hoff;           // [nleaf], law 3 only
  double *d_mat;         // [n_mats][kMatWords]
  float *d_gh;           // warp form: G_p, h_p slots of the resident warps (scratch)
};

namespace dmn {
int material_z_words(int kind) {
  return kind == DMN_MAT_J2_LINEAR ? 7
                                   : (kind == DMN_MAT_J2_PERZYNA ? 13 : (kind == DMN_MAT_PA66 ? kPaZ : 0));
}
int material_hist_words(int kind) { return kind == DMN_MAT_PA66 ? kPaHist : material_z_words(kind); }

// Sec. 4: K = E/(3(1-2nu)), G = E/(2(1+nu)); the device row holds the moduli at
// theta0 and, for the Perzyna leaf, m, 1/t_visc and dE_dT
const char *material_row(const dmn_material &m, double r[kMatWords]) {
  if (m.kind != DMN_MAT_THERMOELASTIC && m.kind != DMN_MAT_J2_LINEAR && m.kind != DMN_MAT_J2_PERZYNA &&
      m.kind != DMN_MAT_PA66)
    return "unknown kind";
  if (!(m.E > 0.0) || !(m.nu > -1.0 && m.nu < 0.5) || !isfinite(m.alpha) || !(m.theta0 > 0.0))
    return "invalid elastic constants";
  for (int i = 0; i < kMatWords; ++i) r[i] = 0.0;
  if (m.kind == DMN_MAT_PA66) {
    if (!(m.sy0 > 0.0) || !(m.k_hard >= 0.0) || !isfinite(m.k_hard) || !(m.n_hard > 0.0 && m.n_hard <= 1.0))
      return "invalid PA66 hardening (sy0 > 0, k_hard >= 0, 0 < n_hard <= 1)";
    if (!(m.m_rate >= 1.0 && m.m_rate <= 8.0) || m.m_rate != floor(m.m_rate) || !(m.eta0 > 0.0) ||
        !isfinite(m.eta0))
      return "invalid PA66 rate law (m an integer in 1..8, eta0 > 0)";
    if (!(m.beta1 >= 0.0) || !isfinite(m.beta1) || !(m.beta2 >= 0.0) || !isfinite(m.beta2) ||
        !(m.theta_ref > 0.0) || !isfinite(m.wlf_C1) || !(m.wlf_C2 > 0.0) || !isfinite(m.wlf_C2))
      return "invalid PA66 softening / WLF constants";
    for (int i = 0; i < kPaBranches; ++i)
      if (!(m.E_maxwell[i] >= 0.0) || !isfinite(m.E_maxwell[i]) ||
          (m.E_maxwell[i] > 0.0 && !(m.tau_maxwell[i] > 0.0 && isfinite(m.tau_maxwell[i]))))
        return "invalid Maxwell branch (E >= 0, tau > 0)";
    r[0] = m.kind;
    r[1] = m.E / (3.0 * (1.0 - 2.0 * m.nu));
    r[2] = m.E / (2.0 * (1.0 + m.nu));
    r[3] = m.alpha;
    r[4] = m.theta0;
    r[5] = m.sy0;
    r[6] = m.k_hard;
    r[7] = m.n_hard;
    r[8] = m.m_rate;
    r[9] = m.eta0;
    r[10] = m.beta1;
    r[11] = m.beta2;
    r[12] = m.theta_ref;
    r[13] = m.wlf_C1;
    r[14] = m.wlf_C2;
    r[15] = m.nu;
    for (int i = 0; i < kPaBranches; ++i) {
      r[16 + i] = m.E_maxwell[i];
      r[28 + i] = m.E_maxwell[i] > 0.0 ? m.tau_maxwell[i] : 1.0;
    }
    return nullptr;
  }
  const bool j2 = m.kind != DMN_MAT_THERMOELASTIC;
  if (j2 && (!(m.sy0 > 0.0) || !isfinite(m.dsy_dT) || !(m.H >= 0.0) || !isfinite(m.H)))
    return "invalid J2 constants";
  const bool vp = m.kind == DMN_MAT_J2_PERZYNA;
  if (vp && (!(m.m_rate >= 1.0 && m.m_rate <= 8.0) || m.m_rate != floor(m.m_rate) ||
             !(m.t_visc > 0.0) || !isfinite(m.t_visc) || !isfinite(m.dE_dT)))
    return "invalid Perzyna constants (m an integer in 1..8, t_visc > 0)";
  r[0] = m.kind;
  r[1] = m.E / (3.0 * (1.0 - 2.0 * m.nu));
  r[2] = m.E / (2.0 * (1.0 + m.nu));
  r[3] = m.alpha;
  r[4] = m.theta0;
  r[5] = j2 ? m.sy0 : 0.0;
  r[6] = j2 ? m.dsy_dT : 0.0;
  r[7] = j2 ? m.H : 0.0;
  r[8] = vp ? m.m_rate : 0.0;
  r[9] = vp ? 1.0 / m.t_visc : 0.0;
  r[10] = vp ? m.dE_dT : 0.0;
  r[11] = 0.0;
  return nullptr;
}

const char *build_tree_tables(int K, const double *leaf_w, const double *normals,
                              const uint8_t *phase_map, const dmn_material *mats, int n_mats,
                              double *mat, double *node, float *node_df, int *zoff, int *hoff,
                              double *wl, TreeLayout *lay, char *why, size_t why_len) {
  const int nleaf = 1 << K, N = nleaf - 1;
  lay->Emax = 0.0;
  for (int i = 0; i < n_mats; ++i) {
    const char *bad = material_row(mats[i], &mat[kMatWords * i]);
    if (bad) {
      snprintf(why, why_len, "material %d (kind %d): %s", i, mats[i].kind, bad);
      return why;
    }
    if (mats[i].E > lay->Emax) lay->Emax = mats[i].E;
  }
  // weights (Sec. 3.1): w > 0, sum 1
  double ws = 0.0;
  for (int j = 0; j < nleaf; ++j) {
    if (!(leaf_w[j] > 0.0) || !isfinite(leaf_w[j])) {
      snprintf(why, why_len, "leaf weight %d is not positive", j);
      return why;
    }
    if (phase_map[j] >= n_mats) {
      snprintf(why, why_len, "phase_map[%d]=%d >= n_mats", j, phase_map[j]);
      return why;
    }
    ws += leaf_w[j];
  }
  if (fabs(ws - 1.0) > 1e-12) {
    snprintf(why, why_len, "weights sum to %.17g", ws);
    return why;
  }
  // node table: n (normalised), c1, c2, w, w c1 c2, 1/(w c1 c2), n/sqrt2;
  // weight propagation bottom-up (Sec. 3.1), the subtree weights of a level
  // replacing those of the level below in place
  for (int j = 0; j < nleaf; ++j) wl[j] = leaf_w[j];
  for (int k = K; k >= 1; --k) {
    const int cnt = 1 << (k - 1);
    for (int i = 0; i < cnt; ++i) {
      const double wa = wl[2 * i], wb = wl[2 * i + 1], w = wa + wb;
      const int p = nleaf - (1 << k) + i;
      const double *nv = normals + 3 * p;
      const double nn = sqrt(nv[0] * nv[0] + nv[1] * nv[1] + nv[2] * nv[2]);
      if (!(nn > 0.0) || !isfinite(nn)) {
        snprintf(why, why_len, "normal %d is zero or not finite", p);
        return why;
      }
      double *r = &node[kNodeWords * p];
      r[0] = nv[0] / nn;
      r[1] = nv[1] / nn;
      r[2] = nv[2] / nn;
      r[3] = wa / w;
      r[4] = 1.0 - r[3];
      r[5] = w;
      r[6] = w * r[3] * r[4];
      r[7] = 1.0 / r[6];
      for (int c = 0; c < 3; ++c) r[8 + c] = r[c] / sqrt(2.0);
      r[11] = 0.0;
      wl[i] = w;  // wl[2i], wl[2i+1] are read before slot i is written
    }
  }
  // float-float node table: (hi, lo) of n, n/sqrt2, c1, c2; then 1/(w c1 c2), w c1 c2
  for (int p = 0; p < N; ++p) {
    const double *r = &node[kNodeWords * p];
    const double v[8] = {r[0], r[1], r[2], r[8], r[9], r[10], r[3], r[4]};
    float *o = &node_df[kNodeDfl * p];
    for (int i = 0; i < kNodeDfl; ++i) o[i] = 0.0f;
    for (int i = 0; i < 8; ++i) {
      const float hi = (float)v[i];
      o[2 * i] = hi;
      o[2 * i + 1] = (float)(v[i] - (double)hi);
    }
    o[16] = (float)r[7];
    o[17] = (float)r[6];
  }
  // z offsets in a state block; with PA66 leaves also the offsets of the
  // leaves' history words in the solve's shared memory
  int off = 8 + 3 * N, law = 1, hw = 0;
  for (int j = 0; j < nleaf; ++j) {
    const int kind = mats[phase_map[j]].kind, zwl = material_z_words(kind);
    if (kind == DMN_MAT_J2_PERZYNA && law < 2) law = 2;
    if (kind == DMN_MAT_PA66) law = 3;
    if (zwl > 0) {
      zoff[j] = off;
      off += zwl;
      hoff[j] = hw;
      hw += material_hist_words(kind);
    } else {
      zoff[j] = -1;
      hoff[j] = -1;
    }
  }
  lay->zend = off;
  lay->zw = off - (8 + 3 * N);
  lay->SW = off + (off & 1);
  lay->law = law;
  lay->hw = hw;
  return nullptr;
}
}  // namespace dmn

static thread_local char g_err[512] = "";

static dmn_status fail(dmn_status s, const char *fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
  return s;
}

static dmn_status cuda_fail(cudaError_t e, const char *what) {
  return fail(e == cudaErrorMemoryAllocation ? DMN_ERR_OOM : DMN_ERR_CUDA, "%s: %s", what,
              cudaGetErrorString(e));
}

extern "C" const char *dmn_last_error(void) { return g_err; }

void dmn::set_error_message(const char *msg) { snprintf(g_err, sizeof(g_err), "%s", msg); }

extern "C" void dmn_default_options(dmn_options *o) {
  if (!o) return;
  memset(o, 0, sizeof(*o));
  o->tol = 1e-10;
  o->gamma = 0.5;
  o->res_floor = 0.0;
  o->maxit = 50;
  o->maxbacktrack = 8;
  o->precision = DMN_PREC_FP64;
}

static void free_handle(dmn_handle h) {
  if (!h) return;
  cudaFree(h->d_node);
  cudaFree(h->d_leafw);
  cudaFree(h->d_node_df);
  cudaFree(h->d_phase);
  cudaFree(h->d_zoff);
  cudaFree(h->d_hoff);
  cudaFree(h->d_mat);
  cudaFree(h->d_queue);
  cudaFree(h->d_open);
  cudaFree(h->d_gh);
  delete h;
}

extern "C" dmn_status dmn_create(dmn_handle *out, int32_t K, const double *leaf_w,
                                 const double *normals, const uint8_t *phase_map,
                                 const dmn_material *mats, int32_t n_mats, const dmn_options *opt) {
  g_err[0] = 0;
  if (!out) return fail(DMN_ERR_ARG, "dmn_create: out is NULL");
  *out = nullptr;
  if (K < 1 || K > 10) return fail(DMN_ERR_ARG, "dmn_create: K=%d outside 1..10", K);
  if (!leaf_w || !normals || !phase_map || !mats)
    return fail(DMN_ERR_ARG, "dmn_create: NULL array argument");
  if (n_mats < 1 || n_mats > kMaxMats)
    return fail(DMN_ERR_ARG, "dmn_create: n_mats=%d outside 1..%d", n_mats, kMaxMats);
  dmn_options o;
  if (opt) o = *opt; else dmn_default_options(&o);
  if (!(o.tol > 0.0) || !(o.gamma > 0.0 && o.gamma < 1.0) || o.maxit < 1 || o.maxbacktrack < 0 ||
      (o.precision != DMN_PREC_FP64 && o.precision != DMN_PREC_MIXED))
    return fail(DMN_ERR_ARG, "dmn_create: invalid options");
  if (!solve_variant_valid(o.solve_variant))
    return fail(DMN_ERR_ARG, "dmn_create: solve_variant %d not in {0, 2, 3, 4, 11, 12, 13, 14, 22, 23, 24}",
                o.solve_variant);
  const int nleaf = 1 << K, N = nleaf - 1;

  // tree setup (Sec. 3.1) and material rows (Sec. 4)
  std::vector<double> mat(kMatWords * n_mats), node(kNodeWords * N), wscr(nleaf);
  std::vector<float> node_df(kNodeDfl * N);
  std::vector<int> zoff(nleaf), hoff(nleaf);
  TreeLayout lay;
  char why[256];
  if (build_tree_tables(K, leaf_w, normals, phase_map, mats, n_mats, mat.data(), node.data(),
                        node_df.data(), zoff.data(), hoff.data(), wscr.data(), &lay, why, sizeof(why)))
    return fail(DMN_ERR_ARG, "dmn_create: %s", why);
  if (!(o.res_floor > 0.0)) o.res_floor = 1e-8 * lay.Emax;
  const int law = lay.law, zend = lay.zend, off = lay.SW;
  int zw = lay.zw;
  if (law == 2 && K > 9) return fail(DMN_ERR_ARG, "dmn_create: Perzyna leaves need K <= 9 (K=%d)", K);
  if (law == 3 && K > 8) return fail(DMN_ERR_ARG, "dmn_create: PA66 leaves need K <= 8 (K=%d)", K);
  if (law == 3) zw = lay.hw;  // the solve keeps the leaves' history, not z, in shared memory
  if (is_warp_variant(o.solve_variant) && !warp_form_supports(K, o.precision == DMN_PREC_MIXED, law))
    return fail(DMN_ERR_ARG,
                "dmn_create: solve_variant %d (one warp per point) needs mixed precision, 6 <= K <= 8 "
                "and thermoelastic / J2 leaves only", o.solve_variant);

  dmn_handle h = new dmn_handle_s();
  memset(h, 0, sizeof(*h));
  h->K = K;
  h->N = N;
  h->nleaf = nleaf;
  h->SW = off;
  h->zend = zend;
  h->n_mats = n_mats;
  h->zw = zw;
  h->law = law;
  h->opt = o;
  cudaError_t e;
  if ((e = cudaGetDevice(&h->device)) != cudaSuccess) { free_handle(h); return cuda_fail(e, "cudaGetDevice"); }
  if ((e = cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device)) != cudaSuccess) {
    free_handle(h);
    return cuda_fail(e, "cudaDeviceGetAttribute");
  }
  const bool mixed = o.precision == DMN_PREC_MIXED;
  {
    int smem_optin = 0;
    cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->device);
    if (solve_smem_bytes(K, zw, n_mats, mixed, o.solve_variant, law) > (size_t)smem_optin) {
      free_handle(h);
      return fail(DMN_ERR_ARG, "dmn_create: K=%d does not fit one SM in the requested precision", K);
    }
    if ((e = prepare_solve(K, zw, n_mats, mixed, o.solve_variant, law, &h->blocks_per_sm)) != cudaSuccess) {
      free_handle(h);
      return cuda_fail(e, "prepare_solve");
    }
    if (h->blocks_per_sm < 1) {
      free_handle(h);
      return fail(DMN_ERR_ARG, "dmn_create: K=%d does not fit one SM in the requested precision", K);
    }
  }
  if ((e = cudaMalloc(&h->d_node, sizeof(double) * kNodeWords * N)) != cudaSuccess ||
      (e = cudaMalloc(&h->d_leafw, sizeof(double) * nleaf)) != cudaSuccess ||
      (e = cudaMalloc(&h->d_node_df, sizeof(float) * kNodeDfl * N)) != cudaSuccess ||
      (e = cudaMalloc(&h->d_phase, nleaf)) != cudaSuccess ||
      (e = cudaMalloc(&h->d_zoff, sizeof(int) * nleaf)) != cudaSuccess ||
      (law == 3 && (e = cudaMalloc(&h->d_hoff, sizeof(int) * nleaf)) != cudaSuccess) ||
      (e = cudaMalloc(&h->d_mat, sizeof(double) * kMatWords * n_mats)) != cudaSuccess ||
      (e = cudaMalloc(&h->d_queue, sizeof(unsigned long long))) != cudaSuccess ||
      (e = cudaMalloc(&h->d_open, sizeof(unsigned long long))) != cudaSuccess ||
      (is_warp_variant(o.solve_variant) &&
       (e = cudaMalloc(&h->d_gh, warp_scratch_bytes_per_cta(K) * size_t(h->num_sms) *
                                     size_t(h->blocks_per_sm))) != cudaSuccess)) {
    free_handle(h);
    return cuda_fail(e, "cudaMalloc");
  }
  if ((e = cudaMemcpy(h->d_node, node.data(), sizeof(double) * kNodeWords * N, cudaMemcpyHostToDevice)) != cudaSuccess ||
      (e = cudaMemcpy(h->d_leafw, leaf_w, sizeof(double) * nleaf, cudaMemcpyHostToDevice)) != cudaSuccess ||
      (e = cudaMemcpy(h->d_node_df, node_df.data(), sizeof(float) * kNodeDfl * N, cudaMemcpyHostToDevice)) != cudaSuccess ||
      (e = cudaMemcpy(h->d_phase, phase_map, nleaf, cudaMemcpyHostToDevice)) != cudaSuccess ||
      (e = cudaMemcpy(h->d_zoff, zoff.data(), sizeof(int) * nleaf, cudaMemcpyHostToDevice)) != cudaSuccess ||
      (law == 3 && (e = cudaMemcpy(h->d_hoff, hoff.data(), sizeof(int) * nleaf, cudaMemcpyHostToDevice)) != cudaSuccess) ||
      (e = cudaMemcpy(h->d_mat, mat.data(), sizeof(double) * kMatWords * n_mats, cudaMemcpyHostToDevice)) != cudaSuccess) {
    free_handle(h);
    return cuda_fail(e, "cudaMemcpy");
  }
  *out = h;
  return DMN_OK;
}

extern "C" dmn_status dmn_destroy(dmn_handle h) {
  g_err[0] = 0;
  if (!h) return fail(DMN_ERR_ARG, "dmn_destroy: NULL handle");
  free_handle(h);
  return DMN_OK;
}

extern "C" int64_t dmn_state_words(dmn_handle h) { return h ? h->SW : -1; }

__global__ void dmn_state_init_kernel(double *s, int64_t n, int SW, const double *theta0) {
  const int64_t total = n * (int64_t)SW;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t pt = i / SW;
    const int w = int(i - pt * SW);
    s[i] = (w == 6) ? theta0[pt] : 0.0;
  }
}

extern "C" dmn_status dmn_state_init(dmn_handle h, double *d_state, int64_t n_points,
                                     const double *d_theta0, dmn_stream stream) {
  g_err[0] = 0;
  if (!h) return fail(DMN_ERR_ARG, "dmn_state_init: NULL handle");
  if (n_points < 0) return fail(DMN_ERR_ARG, "dmn_state_init: n_points < 0");
  if (n_points == 0) return DMN_OK;
  if (!d_state || !d_theta0) return fail(DMN_ERR_ARG, "dmn_state_init: NULL pointer");
  if (((uintptr_t)d_state & 15) != 0) return fail(DMN_ERR_ARG, "dmn_state_init: state not 16-byte aligned");
  const int64_t total = n_points * h->SW;
  int grid = (int)((total + 255) / 256);
  if (grid > 8 * h->num_sms * 8) grid = 8 * h->num_sms * 8;
  dmn_state_init_kernel<<<grid, 256, 0, (cudaStream_t)stream>>>(d_state, n_points, h->SW, d_theta0);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "dmn_state_init launch");
  return DMN_OK;
}

static dmn_status eval_impl(dmn_handle h, dmn_stream stream, int64_t n_points,
                            const double *d_deps, const double *d_theta, double dt,
                            const double *d_state_in, double *d_state_out, double *d_out,
                            int32_t *d_status, int32_t *d_iters, const float *d_da,
                            const int32_t *d_skip = nullptr) {
  g_err[0] = 0;
  if (!h) return fail(DMN_ERR_ARG, "dmn_eval: NULL handle");
  if (n_points < 0) return fail(DMN_ERR_ARG, "dmn_eval: n_points < 0");
  if (n_points == 0) return DMN_OK;
  if (!d_deps || !d_theta || !d_state_in || !d_state_out || !d_out || !d_status || !d_iters)
    return fail(DMN_ERR_ARG, "dmn_eval: NULL pointer");
  if (!(dt > 0.0) || !isfinite(dt)) return fail(DMN_ERR_ARG, "dmn_eval: dt must be > 0");
  if (d_state_in == d_state_out) return fail(DMN_ERR_ARG, "dmn_eval: state_in aliases state_out");
  const size_t sbytes = sizeof(double) * (size_t)h->SW * (size_t)n_points;
  const char *a = (const char *)d_state_in, *b = (const char *)d_state_out;
  if (a < b + sbytes && b < a + sbytes) return fail(DMN_ERR_ARG, "dmn_eval: state_in overlaps state_out");
  if ((((uintptr_t)d_state_in) & 15) || (((uintptr_t)d_state_out) & 15))
    return fail(DMN_ERR_ARG, "dmn_eval: state buffers must be 16-byte aligned");
  const bool mixed = h->opt.precision == DMN_PREC_MIXED;
  SolveParams P;
  memset(&P, 0, sizeof(P));
  P.K = h->K;
  P.N = h->N;
  P.G = 1 << (h->K - 1);
  P.SW = h->SW;
  P.zend = h->zend;
  P.n_mats = h->n_mats;
  P.maxit = h->opt.maxit;
  P.maxbt = h->opt.maxbacktrack;
  P.tol = h->opt.tol;
  P.gamma = h->opt.gamma;
  P.res_floor = h->opt.res_floor;
  P.dt = dt;
  P.node = h->d_node;
  P.leafw = h->d_leafw;
  P.node_df = h->d_node_df;
  P.zw = h->zw;
  P.law = h->law;
  P.phase = h->d_phase;
  P.zoff = h->d_zoff;
  P.hoff = h->d_hoff;
  P.mat = h->d_mat;
  P.n_points = n_points;
  P.deps = d_deps;
  P.theta = d_theta;
  P.sin = d_state_in;
  P.sout = d_state_out;
  P.out = d_out;
  P.status = d_status;
  P.iters = d_iters;
  P.queue = h->d_queue;
  P.da0 = d_da;
  P.skip = d_skip;
  P.gh = h->d_gh;
  int64_t grid = (int64_t)h->num_sms * h->blocks_per_sm;  // the scratch holds this many CTAs
  const int64_t per_cta = is_warp_variant(h->opt.solve_variant) ? warp_form_warps() : 1;
  if (grid > (n_points + per_cta - 1) / per_cta) grid = (n_points + per_cta - 1) / per_cta;
  cudaError_t e = launch_solve(P, mixed, h->opt.solve_variant, (int)grid, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "dmn_eval launch");
  return DMN_OK;
}

extern "C" dmn_status dmn_eval(dmn_handle h, dmn_stream stream, int64_t n_points,
                               const double *d_deps, const double *d_theta, double dt,
                               const double *d_state_in, double *d_state_out, double *d_out,
                               int32_t *d_status, int32_t *d_iters) {
  return eval_impl(h, stream, n_points, d_deps, d_theta, dt, d_state_in, d_state_out, d_out,
                   d_status, d_iters, nullptr);
}

extern "C" dmn_status dmn_eval_warm(dmn_handle h, dmn_stream stream, int64_t n_points,
                                    const double *d_deps, const double *d_theta, double dt,
                                    const double *d_state_in, double *d_state_out, double *d_out,
                                    int32_t *d_status, int32_t *d_iters, const float *d_da) {
  if (!d_da && n_points > 0) return fail(DMN_ERR_ARG, "dmn_eval_warm: d_da is NULL");
  return eval_impl(h, stream, n_points, d_deps, d_theta, dt, d_state_in, d_state_out, d_out,
                   d_status, d_iters, d_da);
}

// Outer Newton of dmn_eval_mixed: evaluate, update the unknown increments and
// temperatures on the device, read back how many points still iterate.
extern "C" dmn_status dmn_eval_mixed(dmn_handle h, dmn_stream stream, int64_t n_points,
                                     const uint8_t *d_mask, const double *d_target, double *d_deps,
                                     double *d_theta, double dt, double c_heat, int32_t max_outer,
                                     double tol_outer, const double *d_state_in,
                                     double *d_state_out, double *d_out, int32_t *d_status,
                                     int32_t *d_iters, int32_t *d_outer, float *d_work,
                                     int32_t flags) {
  g_err[0] = 0;
  if (!h) return fail(DMN_ERR_ARG, "dmn_eval_mixed: NULL handle");
  if (n_points < 0) return fail(DMN_ERR_ARG, "dmn_eval_mixed: n_points < 0");
  if (n_points == 0) return DMN_OK;
  if (!d_mask || !d_target || !d_deps || !d_theta || !d_outer)
    return fail(DMN_ERR_ARG, "dmn_eval_mixed: NULL pointer");
  if (!(c_heat > 0.0) || !isfinite(c_heat)) return fail(DMN_ERR_ARG, "dmn_eval_mixed: c_heat must be > 0");
  if (max_outer < 1) return fail(DMN_ERR_ARG, "dmn_eval_mixed: max_outer must be >= 1");
  if (!(tol_outer > 0.0) || !isfinite(tol_outer))
    return fail(DMN_ERR_ARG, "dmn_eval_mixed: tol_outer must be > 0");
  if (flags & ~DMN_MIXED_PREDICT) return fail(DMN_ERR_ARG, "dmn_eval_mixed: unknown flags");
  if (!d_state_in || !d_out) return fail(DMN_ERR_ARG, "dmn_eval_mixed: NULL pointer");
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = mixed_prepare(s, n_points, h->SW, d_mask, d_target, d_deps, d_theta, dt, c_heat,
                                d_state_in, d_out, (flags & DMN_MIXED_PREDICT) != 0, d_outer);
  if (e != cudaSuccess) return cuda_fail(e, "dmn_eval_mixed prepare");
  for (int it = 0; it < max_outer; ++it) {
    const float *da = (it > 0 && d_work) ? d_work : nullptr;
    // points settled in an earlier evaluation (d_outer != 0) keep its results
    const dmn_status st = eval_impl(h, stream, n_points, d_deps, d_theta, dt, d_state_in,
                                    d_state_out, d_out, d_status, d_iters, da,
                                    it > 0 ? d_outer : nullptr);
    if (st != DMN_OK) return st;
    if ((e = cudaMemsetAsync(h->d_open, 0, sizeof(unsigned long long), s)) != cudaSuccess)
      return cuda_fail(e, "dmn_eval_mixed memset");
    const bool last = it + 1 == max_outer;
    e = mixed_update(s, n_points, h->SW, 3 * h->N, d_mask, d_target, d_deps, d_theta, dt, c_heat,
                     tol_outer, d_state_in, d_state_out, d_out, d_status, d_outer, it, last,
                     last ? nullptr : d_work, h->d_open);
    if (e != cudaSuccess) return cuda_fail(e, "dmn_eval_mixed update");
    if (last) break;
    unsigned long long open = 0;
    if ((e = cudaMemcpyAsync(&open, h->d_open, sizeof(open), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
        (e = cudaStreamSynchronize(s)) != cudaSuccess)
      return cuda_fail(e, "dmn_eval_mixed read-back");
    if (open == 0) break;
  }
  e = mixed_finish(s, n_points, d_status, d_outer);
  if (e != cudaSuccess) return cuda_fail(e, "dmn_eval_mixed finish");
  return DMN_OK;
}

extern "C" dmn_status dmn_debug_bounds_log(int64_t *count, int64_t *index, int64_t *bound, int32_t *line,
                                           int32_t clear) {
  g_err[0] = 0;
  if (!count) return fail(DMN_ERR_ARG, "dmn_debug_bounds_log: count is NULL");
  cudaError_t (*const logs[])(BoundsLog *, bool) = {bounds_log_owner, bounds_log_compact,
                                                    bounds_log_compact_vp, bounds_log_compact_pa66,
                                                    bounds_log_warp, bounds_log_warp8};
  int64_t n = 0;
  bool first = true;
  for (auto f : logs) {
    BoundsLog b;
    const cudaError_t e = f(&b, clear != 0);
    if (e == cudaErrorNotSupported)
      return fail(DMN_ERR_ARG, "dmn_debug_bounds_log: index checks are compiled into the debug library "
                               "(libdmn_debug.so) only");
    if (e != cudaSuccess) return cuda_fail(e, "dmn_debug_bounds_log");
    if (b.count > 0 && first) {
      if (index) *index = b.index;
      if (bound) *bound = b.bound;
      if (line) *line = b.line;
      first = false;
    }
    n += int64_t(b.count);
  }
  *count = n;
  return DMN_OK;
}
