// dmn_linear.cu -- the DMN's linear elastic homogenization function DMN^L and
// the reverse-mode gradient of the offline-training loss (arXiv 2109.14403,
// Sec. 3.2), for a batch of stiffness samples.  Declared in
// include/dmn_linear.h.
//
// dmn_linear_forward: one CTA of G = 2^(K-1) threads per sample, persistent
// over the batch; the laminates of a level run one per thread, the levels one
// after another with a barrier, the node stiffnesses in shared memory.
// dmn_linear_loss_grad: level-synchronous over the whole batch, one launch
// per level and direction, every (sample, node) pair a thread, the node
// stiffnesses and their adjoints in the caller's workspace; the backward pass
// walks the tree top-down: per node it turns the adjoint G of its stiffness
// into the adjoints of its two children and into dJ/dn and dJ/dc1, which each
// block sums over its samples before one FP64 atomic add.
// A laminate is computed in condensed form: with D = C_L - C_R, M = c2 C_L +
// c1 C_R, U = D B, K = B^T M B,
//   C = c1 C_L + c2 C_R - c1 c2 U K^-1 U^T,
// and its reverse mode, with W = U K^-1, A = G W, Q = W^T G W:
//   G_L = c1 G - 2 c1 c2 sym(A B^T) + c1 c2^2 B Q B^T
//   G_R = c2 G + 2 c1 c2 sym(A B^T) + c1^2 c2 B Q B^T
//   dJ/dc1 = <G, D> - (c2 - c1) <U, A> - c1 c2 <Q, B^T U>
//   dJ/dB = -2 c1 c2 (D A - M B Q)
#include <algorithm>
#include <cmath>
#include <cstdio>

#include "../../include/dmn_linear.h"
#include "dmn_internal.h"

namespace dmn {
namespace {

constexpr int kLinMaxK = 8;

// B a = sym(a (x) n): 6x3
template <typename T>
__device__ __forceinline__ void bmat(const T n[3], T B[6][3]) {
  const T r = T(kRsq2);
#pragma unroll
  for (int a = 0; a < 6; ++a)
#pragma unroll
    for (int f = 0; f < 3; ++f) B[a][f] = T(0);
  B[0][0] = n[0];
  B[1][1] = n[1];
  B[2][2] = n[2];
  B[3][1] = r * n[2];
  B[3][2] = r * n[1];
  B[4][0] = r * n[2];
  B[4][2] = r * n[0];
  B[5][0] = r * n[1];
  B[5][1] = r * n[0];
}

// U = D B, MB = M B, K^-1 (symmetric), W = U K^-1
template <typename T>
__device__ __forceinline__ void lam_core(const T *CL, const T *CR, const T B[6][3], T c1, T U[6][3],
                                         T MB[6][3], T Ki[3][3], T W[6][3]) {
  const T c2 = T(1) - c1;
#pragma unroll
  for (int a = 0; a < 6; ++a)
#pragma unroll
    for (int f = 0; f < 3; ++f) {
      T u = T(0), m = T(0);
#pragma unroll
      for (int b = 0; b < 6; ++b) {
        const T l = sget(CL, a, b), r = sget(CR, a, b);
        u += (l - r) * B[b][f];
        m += (c2 * l + c1 * r) * B[b][f];
      }
      U[a][f] = u;
      MB[a][f] = m;
    }
  T Kk[3][3];
#pragma unroll
  for (int e = 0; e < 3; ++e)
#pragma unroll
    for (int f = 0; f < 3; ++f) {
      T s = T(0);
#pragma unroll
      for (int a = 0; a < 6; ++a) s += B[a][e] * MB[a][f];
      Kk[e][f] = s;
    }
  const T k00 = Kk[0][0], k11 = Kk[1][1], k22 = Kk[2][2];
  const T k01 = T(0.5) * (Kk[0][1] + Kk[1][0]), k02 = T(0.5) * (Kk[0][2] + Kk[2][0]);
  const T k12 = T(0.5) * (Kk[1][2] + Kk[2][1]);
  const T a00 = k11 * k22 - k12 * k12, a01 = k02 * k12 - k01 * k22, a02 = k01 * k12 - k02 * k11;
  const T a11 = k00 * k22 - k02 * k02, a12 = k01 * k02 - k00 * k12, a22 = k00 * k11 - k01 * k01;
  const T id = T(1) / (k00 * a00 + k01 * a01 + k02 * a02);
  Ki[0][0] = a00 * id;
  Ki[0][1] = Ki[1][0] = a01 * id;
  Ki[0][2] = Ki[2][0] = a02 * id;
  Ki[1][1] = a11 * id;
  Ki[1][2] = Ki[2][1] = a12 * id;
  Ki[2][2] = a22 * id;
#pragma unroll
  for (int a = 0; a < 6; ++a)
#pragma unroll
    for (int f = 0; f < 3; ++f) W[a][f] = U[a][0] * Ki[0][f] + U[a][1] * Ki[1][f] + U[a][2] * Ki[2][f];
}

template <typename T>
__device__ void lam_forward(const T *CL, const T *CR, const T n[3], T c1, T *out) {
  T B[6][3], U[6][3], MB[6][3], Ki[3][3], W[6][3];
  bmat(n, B);
  lam_core(CL, CR, B, c1, U, MB, Ki, W);
  const T c2 = T(1) - c1, cc = c1 * c2;
#pragma unroll
  for (int i = 0; i < 6; ++i)
#pragma unroll
    for (int j = i; j < 6; ++j) {
      const int q = sidx(i, j);
      out[q] = c1 * CL[q] + c2 * CR[q] - cc * (W[i][0] * U[j][0] + W[i][1] * U[j][1] + W[i][2] * U[j][2]);
    }
}

// reverse mode of one laminate; GL / GR may be null (leaf children)
template <typename T>
__device__ void lam_backward(const T *CL, const T *CR, const T n[3], T c1, const T *G, T *GL, T *GR,
                             T gn[3], T &gc1) {
  T B[6][3], U[6][3], MB[6][3], Ki[3][3], W[6][3];
  bmat(n, B);
  lam_core(CL, CR, B, c1, U, MB, Ki, W);
  const T c2 = T(1) - c1, cc = c1 * c2;
  T A[6][3];
#pragma unroll
  for (int i = 0; i < 6; ++i)
#pragma unroll
    for (int f = 0; f < 3; ++f) {
      T s = T(0);
#pragma unroll
      for (int j = 0; j < 6; ++j) s += sget(G, i, j) * W[j][f];
      A[i][f] = s;
    }
  T Q[3][3];
#pragma unroll
  for (int e = 0; e < 3; ++e)
#pragma unroll
    for (int f = 0; f < 3; ++f) {
      T s = T(0);
#pragma unroll
      for (int i = 0; i < 6; ++i) s += W[i][e] * A[i][f];
      Q[e][f] = s;
    }
#pragma unroll
  for (int e = 0; e < 3; ++e)
#pragma unroll
    for (int f = e + 1; f < 3; ++f) Q[e][f] = Q[f][e] = T(0.5) * (Q[e][f] + Q[f][e]);
  // <G, D>, <U, A>, <Q, B^T U>
  T GD = T(0);
#pragma unroll
  for (int i = 0; i < 6; ++i)
#pragma unroll
    for (int j = i; j < 6; ++j) {
      const int q = sidx(i, j);
      GD += (i == j ? T(1) : T(2)) * G[q] * (CL[q] - CR[q]);
    }
  T UA = T(0), QBU = T(0);
#pragma unroll
  for (int a = 0; a < 6; ++a)
#pragma unroll
    for (int f = 0; f < 3; ++f) UA += U[a][f] * A[a][f];
#pragma unroll
  for (int e = 0; e < 3; ++e)
#pragma unroll
    for (int f = 0; f < 3; ++f) {
      T s = T(0);
#pragma unroll
      for (int a = 0; a < 6; ++a) s += B[a][e] * U[a][f];
      QBU += Q[e][f] * s;
    }
  gc1 = GD - (c2 - c1) * UA - cc * QBU;
  // dJ/dB = -2 c1 c2 (D A - M B Q), then dJ/dn through B(n)
  T gB[6][3];
#pragma unroll
  for (int a = 0; a < 6; ++a)
#pragma unroll
    for (int f = 0; f < 3; ++f) {
      T da = T(0);
#pragma unroll
      for (int b = 0; b < 6; ++b) da += (sget(CL, a, b) - sget(CR, a, b)) * A[b][f];
      const T mbq = MB[a][0] * Q[0][f] + MB[a][1] * Q[1][f] + MB[a][2] * Q[2][f];
      gB[a][f] = T(-2) * cc * (da - mbq);
    }
  const T r = T(kRsq2);
  gn[0] = gB[0][0] + r * (gB[4][2] + gB[5][1]);
  gn[1] = gB[1][1] + r * (gB[3][2] + gB[5][0]);
  gn[2] = gB[2][2] + r * (gB[3][1] + gB[4][0]);
  if (!GL) return;
  T BQ[6][3];
#pragma unroll
  for (int a = 0; a < 6; ++a)
#pragma unroll
    for (int f = 0; f < 3; ++f) BQ[a][f] = B[a][0] * Q[0][f] + B[a][1] * Q[1][f] + B[a][2] * Q[2][f];
#pragma unroll
  for (int i = 0; i < 6; ++i)
#pragma unroll
    for (int j = i; j < 6; ++j) {
      const int q = sidx(i, j);
      const T ab = T(0.5) * (A[i][0] * B[j][0] + A[i][1] * B[j][1] + A[i][2] * B[j][2] + A[j][0] * B[i][0] +
                             A[j][1] * B[i][1] + A[j][2] * B[i][2]);
      const T bqb = BQ[i][0] * B[j][0] + BQ[i][1] * B[j][1] + BQ[i][2] * B[j][2];
      GL[q] = c1 * G[q] - T(2) * cc * ab + cc * c2 * bqb;
      GR[q] = c2 * G[q] + T(2) * cc * ab + cc * c1 * bqb;
    }
}

// shared-memory carving of dmn_linear_forward (T words): normals 3N, c1 N,
// phases 42, nodes 21N
struct LinLayout {
  int nh, c1, ph, ns, words;
};
__host__ __device__ inline LinLayout lin_layout(int K) {
  const int N = (1 << K) - 1;
  LinLayout L;
  L.nh = 0;
  L.c1 = L.nh + 3 * N;
  L.ph = L.c1 + N;
  L.ns = L.ph + 42;
  L.words = L.ns + 21 * N;
  return L;
}

// per-CTA constants: normalised normals, c1 from the weight propagation
// (Sec. 3.1, bottom level first; c1 = W_1 / (W_1 + W_2)).  The subtree
// weights use the node array as scratch (it is free before the first sample);
// ends with a barrier.
template <typename T>
__device__ void lin_constants(int K, const double *normals, const double *v, T *nh, T *c1s, T *scratch) {
  const int N = (1 << K) - 1, L = 1 << K, t = threadIdx.x;
  for (int p = t; p < N; p += blockDim.x) {
    const double x = normals[3 * p], y = normals[3 * p + 1], z = normals[3 * p + 2];
    const double il = 1.0 / sqrt(x * x + y * y + z * z);
    nh[3 * p] = T(x * il);
    nh[3 * p + 1] = T(y * il);
    nh[3 * p + 2] = T(z * il);
  }
  T *Wt = scratch;  // leaves [0, L), nodes [L, L + N)
  for (int j = t; j < L; j += blockDim.x) Wt[j] = T(v[j] > 0.0 ? v[j] : 0.0);
  __syncthreads();
  for (int k = K; k >= 1; --k) {
    for (int i = t; i < (1 << (k - 1)); i += blockDim.x) {
      const int p = (1 << K) - (1 << k) + i;
      const int pc = (1 << K) - (1 << (k + 1)) + 2 * i;
      const T a = k == K ? Wt[2 * i] : Wt[L + pc], b = k == K ? Wt[2 * i + 1] : Wt[L + pc + 1];
      const T W = a + b;
      Wt[L + p] = W;
      c1s[p] = W > T(0) ? a / W : T(0.5);
    }
    __syncthreads();
  }
}

template <typename T>
__device__ void load_phases(const double *C1, const double *C2, T *ph) {
  for (int q = threadIdx.x; q < 42; q += blockDim.x) {
    const double *C = q < 21 ? C1 : C2;
    const int r = q < 21 ? q : q - 21;
    int i = 0, j = 0;
    for (int a = 0, k = 0; a < 6; ++a)
      for (int b = a; b < 6; ++b, ++k)
        if (k == r) {
          i = a;
          j = b;
        }
    ph[q] = T(0.5 * (C[6 * i + j] + C[6 * j + i]));
  }
}

// bottom-up pass of one sample into the node array
template <typename T>
__device__ void lin_sweep_up(int K, const T *nh, const T *c1s, const T *ph, T *ns) {
  for (int k = K; k >= 1; --k) {
    const int cnt = 1 << (k - 1);
    for (int j = threadIdx.x; j < cnt; j += blockDim.x) {
      const int p = (1 << K) - (1 << k) + j;
      const T *CL, *CR;
      if (k == K) {
        CL = ph;
        CR = ph + 21;
      } else {
        const int pc = (1 << K) - (1 << (k + 1)) + 2 * j;
        CL = ns + 21 * pc;
        CR = ns + 21 * (pc + 1);
      }
      lam_forward(CL, CR, nh + 3 * p, c1s[p], ns + 21 * p);
    }
    __syncthreads();
  }
}

// per-sample error e_s = |T - D|_p / |T|_p over the 36 components (FP64)
template <typename T>
__device__ double lin_error(const double *Tg, const T *D, double p) {
  double num = 0.0, den = 0.0;
  for (int i = 0; i < 6; ++i)
    for (int j = 0; j < 6; ++j) {
      const double x = Tg[6 * i + j] - double(sget(D, i, j)), y = Tg[6 * i + j];
      num += pow(fabs(x), p);
      den += pow(fabs(y), p);
    }
  return pow(num, 1.0 / p) / pow(den, 1.0 / p);
}

template <typename T>
__global__ void k_lin_forward(int K, int64_t n, const double *C1, const double *C2, const double *normals,
                              const double *v, const double *Ctarget, double p, double *Cbar,
                              double *err) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *sm = reinterpret_cast<T *>(smem_raw);
  const LinLayout L = lin_layout(K);
  const int N = (1 << K) - 1, root = N - 1;
  lin_constants<T>(K, normals, v, sm + L.nh, sm + L.c1, sm + L.ns);
  for (int64_t s = blockIdx.x; s < n; s += gridDim.x) {
    load_phases<T>(C1 + 36 * s, C2 + 36 * s, sm + L.ph);
    __syncthreads();
    lin_sweep_up<T>(K, sm + L.nh, sm + L.c1, sm + L.ph, sm + L.ns);
    const T *D = sm + L.ns + 21 * root;
    if (Cbar)
      for (int q = threadIdx.x; q < 36; q += blockDim.x) Cbar[36 * s + q] = double(sget(D, q / 6, q % 6));
    if (err && threadIdx.x == 0) err[s] = lin_error<T>(Ctarget + 36 * s, D, p);
    __syncthreads();
  }
}

// batch reduction of the errors: scal[0] = max e, scal[1] = (1/N) S^(1/q - 1)
// with S = sum (e/max)^q, scal[2] = data term; also the penalty and J
__global__ void k_lin_reduce(int K, int64_t n, const double *err, const double *v, double q, double penalty,
                             double *scal, double *loss) {
  __shared__ double red[1024];
  const int t = threadIdx.x;
  double m = 0.0;
  for (int64_t s = t; s < n; s += blockDim.x) m = fmax(m, err[s]);
  red[t] = m;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (t < o) red[t] = fmax(red[t], red[t + o]);
    __syncthreads();
  }
  m = red[0];
  __syncthreads();
  double acc = 0.0;
  if (m > 0.0)
    for (int64_t s = t; s < n; s += blockDim.x) acc += pow(err[s] / m, q);
  red[t] = acc;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (t < o) red[t] += red[t + o];
    __syncthreads();
  }
  if (t == 0) {
    const double S = red[0];
    double wsum = 0.0;
    for (int j = 0; j < (1 << K); ++j) wsum += v[j] > 0.0 ? v[j] : 0.0;
    const double data = m > 0.0 ? m * pow(S, 1.0 / q) / double(n) : 0.0;
    const double pen = penalty * (wsum - 1.0) * (wsum - 1.0);
    scal[0] = m;
    scal[1] = m > 0.0 ? pow(S, 1.0 / q - 1.0) / double(n) : 0.0;
    scal[2] = data;
    loss[0] = data + pen;
    loss[1] = data;
    loss[2] = pen;
  }
}

// ---- level-synchronous training pass over the whole batch.  Node values
// live in the caller's workspace as [node][21][sample] (samples fastest, so a
// warp's loads of one component are contiguous); one launch per level and
// direction, a 2-D grid of (sample blocks, nodes of the level), so every
// block serves one node and reduces its gradient terms before one atomic add.
constexpr int kLvlThreads = 128;

template <typename T>
__device__ __forceinline__ void lvl_load(const T *X, int p, int64_t n, int64_t s, T out[21]) {
#pragma unroll
  for (int q = 0; q < 21; ++q) out[q] = X[(int64_t(p) * 21 + q) * n + s];
}
template <typename T>
__device__ __forceinline__ void lvl_store(T *X, int p, int64_t n, int64_t s, const T v[21]) {
#pragma unroll
  for (int q = 0; q < 21; ++q) X[(int64_t(p) * 21 + q) * n + s] = v[q];
}
template <typename T>
__device__ __forceinline__ void phase_packed(const double *C, T out[21]) {
#pragma unroll
  for (int i = 0; i < 6; ++i)
#pragma unroll
    for (int j = i; j < 6; ++j) out[sidx(i, j)] = T(0.5 * (C[6 * i + j] + C[6 * j + i]));
}

// normalised normals and c1 of every node in the laminate precision (one CTA)
template <typename T>
__global__ void k_lvl_const(int K, const double *normals, const double *v, T *nh, T *c1s) {
  __shared__ double Wt[2 * (1 << kLinMaxK)];
  const int N = (1 << K) - 1, L = 1 << K, t = threadIdx.x;
  for (int pp = t; pp < N; pp += blockDim.x) {
    const double x = normals[3 * pp], y = normals[3 * pp + 1], z = normals[3 * pp + 2];
    const double il = 1.0 / sqrt(x * x + y * y + z * z);
    nh[3 * pp] = T(x * il);
    nh[3 * pp + 1] = T(y * il);
    nh[3 * pp + 2] = T(z * il);
  }
  for (int j = t; j < L; j += blockDim.x) Wt[j] = v[j] > 0.0 ? v[j] : 0.0;
  __syncthreads();
  for (int k = K; k >= 1; --k) {
    for (int i = t; i < (1 << (k - 1)); i += blockDim.x) {
      const int pp = (1 << K) - (1 << k) + i;
      const int pc = (1 << K) - (1 << (k + 1)) + 2 * i;
      const double a = k == K ? Wt[2 * i] : Wt[L + pc], b = k == K ? Wt[2 * i + 1] : Wt[L + pc + 1];
      const double W = a + b;
      Wt[L + pp] = W;
      c1s[pp] = T(W > 0.0 ? a / W : 0.5);
    }
    __syncthreads();
  }
}

// the phase stiffnesses of every sample, packed, in the laminate precision:
// PH[phase][21][sample] (converted once instead of by every bottom laminate)
template <typename T>
__global__ void k_lvl_phases(int64_t n, const double *C1, const double *C2, T *PH) {
  const int64_t s = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (s >= n) return;
  T a[21], b[21];
  phase_packed(C1 + 36 * s, a);
  phase_packed(C2 + 36 * s, b);
  lvl_store(PH, 0, n, s, a);
  lvl_store(PH, 1, n, s, b);
}

template <typename T>
__global__ void __launch_bounds__(kLvlThreads) k_lvl_fwd(int K, int k, int64_t n, const T *PH, const T *nh,
                                                         const T *c1s, T *NS) {
  const int64_t s = int64_t(blockIdx.x) * kLvlThreads + threadIdx.x;
  if (s >= n) return;
  const int j = blockIdx.y, pp = (1 << K) - (1 << k) + j;
  T CL[21], CR[21], out[21];
  if (k == K) {
    lvl_load(PH, 0, n, s, CL);
    lvl_load(PH, 1, n, s, CR);
  } else {
    const int pc = (1 << K) - (1 << (k + 1)) + 2 * j;
    lvl_load(NS, pc, n, s, CL);
    lvl_load(NS, pc + 1, n, s, CR);
  }
  const T nn[3] = {nh[3 * pp], nh[3 * pp + 1], nh[3 * pp + 2]};
  lam_forward(CL, CR, nn, c1s[pp], out);
  lvl_store(NS, pp, n, s, out);
}

// per-sample error from the root column
template <typename T>
__global__ void k_lvl_err(int K, int64_t n, const T *NS, const double *Ct, double p, double *err) {
  const int64_t s = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (s >= n) return;
  T D[21];
  lvl_load(NS, (1 << K) - 2, n, s, D);
  err[s] = lin_error<T>(Ct + 36 * s, D, p);
}

// dJ/dD at the root: (1/N) S^(1/q-1) (e_s/m)^(q-1) de_s/dD
template <typename T>
__global__ void k_lvl_seed(int K, int64_t n, const T *NS, const double *Ct, double p, double q, const double *err,
                           const double *scal, T *GA) {
  const int64_t s = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (s >= n) return;
  const int root = (1 << K) - 2;
  T D[21], G[21];
  lvl_load(NS, root, n, s, D);
  const double m = scal[0], e = err[s];
  const double coef = (m > 0.0 && e > 0.0) ? scal[1] * pow(e / m, q - 1.0) : 0.0;
  const double *Tg = Ct + 36 * s;
  double num = 0.0, den = 0.0;
  for (int i = 0; i < 36; ++i) {
    num += pow(fabs(Tg[i] - double(sget(D, i / 6, i % 6))), p);
    den += pow(fabs(Tg[i]), p);
  }
  const double nx = pow(num, 1.0 / p), nt = pow(den, 1.0 / p);
  for (int i = 0; i < 6; ++i)
    for (int j = i; j < 6; ++j) {
      const double x = Tg[6 * i + j] - double(sget(D, i, j));
      const double sg = x > 0.0 ? 1.0 : (x < 0.0 ? -1.0 : 0.0);
      const double de = nx > 0.0 ? -sg * pow(fabs(x), p - 1.0) * pow(nx, 1.0 - p) / nt : 0.0;
      G[sidx(i, j)] = T(coef * de);
    }
  lvl_store(GA, root, n, s, G);
}

template <typename T>
__global__ void __launch_bounds__(kLvlThreads) k_lvl_bwd(int K, int k, int64_t n, const T *PH, const T *nh,
                                                         const T *c1s, const T *NS, T *GA, double *gnh,
                                                         double *gc1) {
  __shared__ T red[4][kLvlThreads / 32];
  const int64_t s = int64_t(blockIdx.x) * kLvlThreads + threadIdx.x;
  const int j = blockIdx.y, pp = (1 << K) - (1 << k) + j;
  T gn[3] = {T(0), T(0), T(0)}, g1 = T(0);
  if (s < n) {
    T CL[21], CR[21], G[21], GL[21], GR[21];
    const int pc = (1 << K) - (1 << (k + 1)) + 2 * j;
    if (k == K) {
      lvl_load(PH, 0, n, s, CL);
      lvl_load(PH, 1, n, s, CR);
    } else {
      lvl_load(NS, pc, n, s, CL);
      lvl_load(NS, pc + 1, n, s, CR);
    }
    lvl_load(GA, pp, n, s, G);
    const T nn[3] = {nh[3 * pp], nh[3 * pp + 1], nh[3 * pp + 2]};
    lam_backward(CL, CR, nn, c1s[pp], G, k < K ? GL : nullptr, k < K ? GR : nullptr, gn, g1);
    if (k < K) {
      lvl_store(GA, pc, n, s, GL);
      lvl_store(GA, pc + 1, n, s, GR);
    }
  }
  // block sums of dJ/dn and dJ/dc1 of this node (laminate precision), one
  // FP64 atomic add each
  T r[4] = {gn[0], gn[1], gn[2], g1};
#pragma unroll
  for (int c = 0; c < 4; ++c)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) r[c] += __shfl_down_sync(0xffffffffu, r[c], o);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0)
#pragma unroll
    for (int c = 0; c < 4; ++c) red[c][warp] = r[c];
  __syncthreads();
  if (threadIdx.x < 4) {
    T acc = T(0);
    for (int w = 0; w < kLvlThreads / 32; ++w) acc += red[threadIdx.x][w];
    atomicAdd(threadIdx.x < 3 ? gnh + 3 * pp + threadIdx.x : gc1 + pp, double(acc));
  }
}

// the chain through the weights (c1 = W_1 / W, w = <v>_+, penalty) and the
// normalisation of the normals; one thread
__global__ void k_lin_finish(int K, const double *normals, const double *v, double penalty, const double *gnh,
                             const double *gc1, double *grad_n, double *grad_v) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const int N = (1 << K) - 1, L = 1 << K;
  for (int pp = 0; pp < N; ++pp) {
    const double x = normals[3 * pp], y = normals[3 * pp + 1], z = normals[3 * pp + 2];
    const double len = sqrt(x * x + y * y + z * z);
    const double nh[3] = {x / len, y / len, z / len};
    const double g[3] = {gnh[3 * pp], gnh[3 * pp + 1], gnh[3 * pp + 2]};
    const double gd = g[0] * nh[0] + g[1] * nh[1] + g[2] * nh[2];
    for (int c = 0; c < 3; ++c) grad_n[3 * pp + c] = (g[c] - gd * nh[c]) / len;
  }
  // subtree weights of every node, bottom level first
  double Wn[(1 << kLinMaxK) - 1];
  double wsum = 0.0;
  for (int j = 0; j < L; ++j) wsum += v[j] > 0.0 ? v[j] : 0.0;
  for (int k = K; k >= 1; --k)
    for (int i = 0; i < (1 << (k - 1)); ++i) {
      const int pp = (1 << K) - (1 << k) + i;
      double a, b;
      if (k == K) {
        a = v[2 * i] > 0.0 ? v[2 * i] : 0.0;
        b = v[2 * i + 1] > 0.0 ? v[2 * i + 1] : 0.0;
      } else {
        const int pc = (1 << K) - (1 << (k + 1)) + 2 * i;
        a = Wn[pc];
        b = Wn[pc + 1];
      }
      Wn[pp] = a + b;
    }
  // adjoints of the subtree weights, root first
  double gW[(1 << kLinMaxK) - 1];
  gW[N - 1] = 2.0 * penalty * (wsum - 1.0);
  for (int k = 1; k <= K; ++k)
    for (int i = 0; i < (1 << (k - 1)); ++i) {
      const int pp = (1 << K) - (1 << k) + i;
      const double W = Wn[pp];
      double a, b;
      if (k == K) {
        a = v[2 * i] > 0.0 ? v[2 * i] : 0.0;
        b = v[2 * i + 1] > 0.0 ? v[2 * i + 1] : 0.0;
      } else {
        const int pc = (1 << K) - (1 << (k + 1)) + 2 * i;
        a = Wn[pc];
        b = Wn[pc + 1];
      }
      const double dL = W > 0.0 ? gc1[pp] * b / (W * W) : 0.0;   // d c1 / d W_1 = W_2 / W^2
      const double dR = W > 0.0 ? -gc1[pp] * a / (W * W) : 0.0;  // d c1 / d W_2 = -W_1 / W^2
      if (k == K) {
        grad_v[2 * i] = v[2 * i] > 0.0 ? gW[pp] + dL : 0.0;
        grad_v[2 * i + 1] = v[2 * i + 1] > 0.0 ? gW[pp] + dR : 0.0;
      } else {
        const int pc = (1 << K) - (1 << (k + 1)) + 2 * i;
        gW[pc] = gW[pp] + dL;
        gW[pc + 1] = gW[pp] + dR;
      }
    }
}

__global__ void k_lin_zero(double *x, int64_t n) {
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    x[i] = 0.0;
}

__global__ void k_amsgrad(int64_t n, double *x, const double *g, double *m, double *s, double *smax, double lr,
                          double b1, double b2, double eps, double c1, double c2) {
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
    m[i] = b1 * m[i] + (1.0 - b1) * g[i];
    s[i] = b2 * s[i] + (1.0 - b2) * g[i] * g[i];
    smax[i] = fmax(smax[i], s[i]);
    x[i] -= lr * (m[i] / c1) / (sqrt(smax[i] / c2) + eps);
  }
}

dmn_status lin_fail(const char *msg) {
  set_error_message(msg);
  return DMN_ERR_ARG;
}

dmn_status lin_cuda(cudaError_t e, const char *what) {
  char msg[256];
  snprintf(msg, sizeof(msg), "%s: %s", what, cudaGetErrorString(e));
  set_error_message(msg);
  return DMN_ERR_CUDA;
}

// grid of a persistent launch: resident CTAs on every SM, at most n
template <typename Kern>
cudaError_t lin_grid(Kern f, int threads, size_t smem, int64_t n, int *grid) {
  int dev = 0, sms = 0, per = 0;
  cudaError_t e;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  if ((e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem))) != cudaSuccess)
    return e;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, f, threads, smem)) != cudaSuccess) return e;
  if (per < 1) return cudaErrorInvalidConfiguration;
  const int64_t g = std::min<int64_t>(int64_t(sms) * per, n);
  *grid = int(std::max<int64_t>(g, 1));
  return cudaSuccess;
}

const char *lin_check(int32_t K, int64_t n, const double *C1, const double *C2, const double *normals,
                      const double *v, int32_t precision) {
  if (K < 1 || K > kLinMaxK) return "K must be 1..8";
  if (n < 0) return "n_samples < 0";
  if (n > 0 && (!C1 || !C2 || !normals || !v)) return "NULL pointer";
  if (precision != DMN_LIN_FP64 && precision != DMN_LIN_FP32) return "unknown precision";
  return nullptr;
}

template <typename T>
dmn_status lin_forward(cudaStream_t st, int K, int64_t n, const double *C1, const double *C2,
                       const double *normals, const double *v, const double *Ct, double p, double *Cbar,
                       double *err) {
  const size_t smem = sizeof(T) * lin_layout(K).words;
  const int threads = 1 << (K - 1);
  int grid = 0;
  cudaError_t e = lin_grid(k_lin_forward<T>, threads, smem, n, &grid);
  if (e != cudaSuccess) return lin_cuda(e, "dmn_linear: launch configuration");
  k_lin_forward<T><<<grid, threads, smem, st>>>(K, n, C1, C2, normals, v, Ct, p, Cbar, err);
  if ((e = cudaGetLastError()) != cudaSuccess) return lin_cuda(e, "dmn_linear: forward launch");
  return DMN_OK;
}

// the training pass: forward by levels, errors, batch reduction, seed,
// backward by levels; NS and GA in the workspace
template <typename T>
dmn_status lin_train_pass(cudaStream_t st, int K, int64_t n, const double *C1, const double *C2,
                          const double *Ct, const double *normals, const double *v, double p, double q,
                          double penalty, double *err, double *scal, double *loss, T *consts, T *PH, T *NS, T *GA,
                          double *gnh, double *gc1) {
  const unsigned nb = unsigned((n + kLvlThreads - 1) / kLvlThreads);
  if (nb > 2147483647u) return lin_fail("dmn_linear_loss_grad: batch too large");
  const int N = (1 << K) - 1;
  T *nh = consts, *c1s = consts + 3 * N;
  k_lvl_const<T><<<1, 256, 0, st>>>(K, normals, v, nh, c1s);
  k_lvl_phases<T><<<nb, kLvlThreads, 0, st>>>(n, C1, C2, PH);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return lin_cuda(e, "dmn_linear: set-up launch");
  for (int k = K; k >= 1; --k) {
    k_lvl_fwd<T><<<dim3(nb, 1u << (k - 1)), kLvlThreads, 0, st>>>(K, k, n, PH, nh, c1s, NS);
    if ((e = cudaGetLastError()) != cudaSuccess) return lin_cuda(e, "dmn_linear: forward level launch");
  }
  k_lvl_err<T><<<nb, kLvlThreads, 0, st>>>(K, n, NS, Ct, p, err);
  k_lin_reduce<<<1, 1024, 0, st>>>(K, n, err, v, q, penalty, scal, loss);
  k_lvl_seed<T><<<nb, kLvlThreads, 0, st>>>(K, n, NS, Ct, p, q, err, scal, GA);
  if ((e = cudaGetLastError()) != cudaSuccess) return lin_cuda(e, "dmn_linear: loss launch");
  for (int k = 1; k <= K; ++k) {
    k_lvl_bwd<T><<<dim3(nb, 1u << (k - 1)), kLvlThreads, 0, st>>>(K, k, n, PH, nh, c1s, NS, GA, gnh, gc1);
    if ((e = cudaGetLastError()) != cudaSuccess) return lin_cuda(e, "dmn_linear: backward level launch");
  }
  return DMN_OK;
}

}  // namespace
}  // namespace dmn

using namespace dmn;

extern "C" dmn_status dmn_linear_forward(dmn_stream stream, int32_t K, int64_t n_samples, const double *d_C1,
                                         const double *d_C2, const double *d_normals, const double *d_v,
                                         double *d_Cbar, int32_t precision) {
  set_error_message("");
  if (const char *why = lin_check(K, n_samples, d_C1, d_C2, d_normals, d_v, precision)) return lin_fail(why);
  if (n_samples > 0 && !d_Cbar) return lin_fail("dmn_linear_forward: NULL output");
  if (n_samples == 0) return DMN_OK;
  cudaStream_t st = (cudaStream_t)stream;
  return precision == DMN_LIN_FP64
             ? lin_forward<double>(st, K, n_samples, d_C1, d_C2, d_normals, d_v, nullptr, 1.0, d_Cbar, nullptr)
             : lin_forward<float>(st, K, n_samples, d_C1, d_C2, d_normals, d_v, nullptr, 1.0, d_Cbar, nullptr);
}

extern "C" dmn_status dmn_linear_loss_grad(dmn_stream stream, int32_t K, int64_t n_samples, const double *d_C1,
                                           const double *d_C2, const double *d_Ctarget, const double *d_normals,
                                           const double *d_v, double p, double q, double penalty,
                                           double *d_loss, double *d_grad_n, double *d_grad_v, double *d_work,
                                           int32_t precision) {
  set_error_message("");
  if (const char *why = lin_check(K, n_samples, d_C1, d_C2, d_normals, d_v, precision)) return lin_fail(why);
  if (n_samples < 1) return lin_fail("dmn_linear_loss_grad: needs at least one sample");
  if (!d_Ctarget || !d_loss || !d_grad_n || !d_grad_v || !d_work)
    return lin_fail("dmn_linear_loss_grad: NULL pointer");
  if (!(p >= 1.0) || !(q >= 1.0) || !std::isfinite(p) || !std::isfinite(q) || !(penalty >= 0.0) ||
      !std::isfinite(penalty))
    return lin_fail("dmn_linear_loss_grad: p, q >= 1 and penalty >= 0 required");
  cudaStream_t st = (cudaStream_t)stream;
  const int N = (1 << K) - 1;
  double *err = d_work, *gnh = d_work + n_samples, *gc1 = gnh + 3 * N, *scal = gc1 + N;
  double *consts = scal + 8, *nodes = consts + 4 * N;
  k_lin_zero<<<8, 256, 0, st>>>(gnh, 4 * N + 8);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return lin_cuda(e, "dmn_linear: set-up launch");
  const int64_t cells = int64_t(21) * N * n_samples, ph = int64_t(42) * n_samples;
  dmn_status s;
  if (precision == DMN_LIN_FP64)
    s = lin_train_pass<double>(st, K, n_samples, d_C1, d_C2, d_Ctarget, d_normals, d_v, p, q, penalty, err, scal,
                               d_loss, consts, nodes, nodes + ph, nodes + ph + cells, gnh, gc1);
  else {
    float *f = reinterpret_cast<float *>(nodes);
    s = lin_train_pass<float>(st, K, n_samples, d_C1, d_C2, d_Ctarget, d_normals, d_v, p, q, penalty, err, scal,
                              d_loss, reinterpret_cast<float *>(consts), f, f + ph, f + ph + cells, gnh, gc1);
  }
  if (s != DMN_OK) return s;
  k_lin_finish<<<1, 32, 0, st>>>(K, d_normals, d_v, penalty, gnh, gc1, d_grad_n, d_grad_v);
  if ((e = cudaGetLastError()) != cudaSuccess) return lin_cuda(e, "dmn_linear: finish launch");
  return DMN_OK;
}

extern "C" dmn_status dmn_linear_amsgrad(dmn_stream stream, int64_t n_params, double *d_params,
                                         const double *d_grad, double *d_m, double *d_s, double *d_smax, double lr,
                                         double beta1, double beta2, double eps, int64_t step) {
  set_error_message("");
  if (n_params < 0 || step < 1) return lin_fail("dmn_linear_amsgrad: n_params >= 0 and step >= 1 required");
  if (n_params == 0) return DMN_OK;
  if (!d_params || !d_grad || !d_m || !d_s || !d_smax) return lin_fail("dmn_linear_amsgrad: NULL pointer");
  if (!(beta1 >= 0.0 && beta1 < 1.0) || !(beta2 >= 0.0 && beta2 < 1.0) || !(eps > 0.0) || !std::isfinite(lr))
    return lin_fail("dmn_linear_amsgrad: 0 <= beta < 1, eps > 0 required");
  const double c1 = 1.0 - std::pow(beta1, double(step)), c2 = 1.0 - std::pow(beta2, double(step));
  const int blocks = int(std::min<int64_t>((n_params + 255) / 256, 1024));
  k_amsgrad<<<blocks, 256, 0, (cudaStream_t)stream>>>(n_params, d_params, d_grad, d_m, d_s, d_smax, lr, beta1,
                                                      beta2, eps, c1, c2);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return lin_cuda(e, "dmn_linear_amsgrad launch");
  return DMN_OK;
}
