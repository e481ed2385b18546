// mlp.cu -- the warm-start network of include/dmn_mlp.h: tensor maps, the
// tcgen05 GEMM launches of the forward and backward passes, and the small
// memory-bound kernels around them (features, normalisation, loss, bias
// gradients, AMSGrad, weight packing, transposes).
#include <cudaTypedefs.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <vector>

#include "../../include/dmn.h"
#include "../../include/dmn_mlp.h"
#include "dmn_internal.h"
#include "mlp_gemm.cuh"

using namespace dmn;
using namespace dmn::mlp;
typedef __nv_bfloat16 bf16;

namespace {

// ------------------------------------------------------------------ TMA maps
PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;

cudaError_t get_encode() {
  if (g_encode) return cudaSuccess;
  cudaDriverEntryPointQueryResult q;
  void *fn = nullptr;
  cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000,
                                                   cudaEnableDefault, &q);
  if (e != cudaSuccess) return e;
  if (q != cudaDriverEntryPointSuccess || !fn) return cudaErrorNotSupported;
  g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  return cudaSuccess;
}

// bf16 row-major [rows x cols] read in box_rows x 64-column boxes, 128 B swizzle
bool make_map(CUtensorMap *map, const void *ptr, uint64_t rows, uint64_t cols, uint32_t box_rows = 128) {
  const cuuint64_t dims[2] = {cols, rows};
  const cuuint64_t strides[1] = {cols * 2};
  const cuuint32_t box[2] = {64, box_rows};
  const cuuint32_t es[2] = {1, 1};
  return g_encode(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(ptr), dims, strides,
                  box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

int g_gemm_configured_dev = -1;
int g_gemm_sms = 0;

// C = A . B^T with the fused epilogue ep; A [M x K], B [N x K] bf16.  N a
// multiple of 256: the persistent wide form (one CTA per SM), else the tile
// form.
cudaError_t gemm(cudaStream_t s, const void *A, const void *B, int M, int N, int K, EpiArgs ep) {
  if (M % BM || N % BN || K % BK || M <= 0 || N <= 0 || K <= 0) return cudaErrorInvalidValue;
  if (M / BM > 65535 || N / BN > 65535) return cudaErrorInvalidValue;  // grid limits
  if ((reinterpret_cast<uintptr_t>(A) | reinterpret_cast<uintptr_t>(B)) & 15) return cudaErrorInvalidValue;
  cudaError_t e = get_encode();
  if (e != cudaSuccess) return e;
  int dev = 0;
  cudaGetDevice(&dev);
  if (g_gemm_configured_dev != dev) {
    e = cudaFuncSetAttribute(gemm_bf16_tn, cudaFuncAttributeMaxDynamicSharedMemorySize, GEMM_SMEM);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(gemm_bf16_tn_wide, cudaFuncAttributeMaxDynamicSharedMemorySize, WGEMM_SMEM);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&g_gemm_sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    g_gemm_configured_dev = dev;
  }
  CUtensorMap ma, mb;
  if (N % WBN == 0) {
    if (!make_map(&ma, A, M, K) || !make_map(&mb, B, N, K, WBN)) return cudaErrorInvalidValue;
    const int tiles = (M / BM) * (N / WBN);
    gemm_bf16_tn_wide<<<tiles < g_gemm_sms ? tiles : g_gemm_sms, 64 + 32 * WEPI, WGEMM_SMEM, s>>>(ma, mb, M, N,
                                                                                              K, ep);
    return cudaGetLastError();
  }
  if (!make_map(&ma, A, M, K) || !make_map(&mb, B, N, K)) return cudaErrorInvalidValue;
  gemm_bf16_tn<<<dim3(N / BN, M / BM), 128, GEMM_SMEM, s>>>(ma, mb, K, ep);
  return cudaGetLastError();
}

int64_t rup(int64_t x, int64_t m) { return (x + m - 1) / m * m; }
unsigned blocks_for(int64_t n, int t = 256) {
  int64_t b = (n + t - 1) / t;
  return unsigned(b < 1 ? 1 : (b > 65535 * 8 ? 65535 * 8 : b));
}

// ------------------------------------------------------------------ kernels
// A double rounded to the nearest float (ties to even) by integer
// operations: the FP64 pipe of this GPU runs at 1/64 of the FP32 rate, and
// the network input converts 768 words per row.  Magnitudes outside the
// normal float range (and NaN) take the FP64 conversion; zero and double
// subnormals give a signed zero.
__device__ __forceinline__ float f32_rn(double d) {
  const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(d));
  const unsigned E = unsigned(b >> 52) & 0x7ffu;
  const unsigned sign = unsigned(b >> 32) & 0x80000000u;
  if (E == 0u) return __uint_as_float(sign);
  if (E < 897u || E > 1150u) return __double2float_rn(d);
  const unsigned long long mant = b & ((1ull << 52) - 1);
  unsigned r = sign | ((E - 896u) << 23) | unsigned(mant >> 29);
  const unsigned rem = unsigned(mant & ((1ull << 29) - 1)), half = 1u << 28;
  if (rem > half || (rem == half && (r & 1u))) r += 1u;  // a carry moves into the exponent
  return __uint_as_float(r);
}

// feature c of a row: deps (6), theta^{n+1}, theta^{n+1} - theta^n,
// a^n - a^{n-1} (n3) as the difference of the two words rounded to float;
// a = the state block at t^n, ap = at t^{n-1} or NULL (its columns 0)
constexpr int kExtraFeatures = 0;
__device__ __forceinline__ float feature(int c, int n3, const double *dep, double th, const double *a,
                                         const double *ap) {
  (void)n3;
  if (c < 6) return f32_rn(dep[c]);
  if (c == 6) return f32_rn(th);
  if (c == 7) return float(th - a[6]);
  return ap ? f32_rn(a[c]) - f32_rn(ap[c]) : 0.0f;  // a^n - a^{n-1}: state words 8..
}

__global__ void k_features(int64_t n, int n3, int sw, const double *deps, const double *theta,
                           const double *sin, const double *sprev, float *feat) {
  const int nin = 8 + n3 + kExtraFeatures;
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n * nin;
       i += int64_t(gridDim.x) * blockDim.x) {
    const int64_t r = i / nin;
    const int c = int(i - r * nin);
    feat[i] = feature(c, n3, deps + r * 6, theta[r], sin + r * sw, sprev ? sprev + r * sw : nullptr);
  }
}

// features of k_features, normalised and rounded to bf16 in one pass: one
// warp per row, each lane two adjacent columns per step (one bf16x2 store;
// ld = kin is a multiple of 128, so the pairs stay 4-byte aligned)
__global__ void k_features_norm(int64_t n, int n3, int sw, int ld, const double *deps,
                                const double *theta, const double *sin, const double *sprev,
                                const float *mean, const float *inv, bf16 *x) {
  const int nin = 8 + n3 + kExtraFeatures;
  const int lane = threadIdx.x & 31;
  const int64_t nwarp = (int64_t(gridDim.x) * blockDim.x) >> 5;
  for (int64_t r = (blockIdx.x * int64_t(blockDim.x) + threadIdx.x) >> 5; r < n; r += nwarp) {
    const double *a = sin + r * sw;
    const double *ap = sprev ? sprev + r * sw : nullptr;
    __nv_bfloat162 *xr = reinterpret_cast<__nv_bfloat162 *>(x + r * ld);
    for (int c0 = 2 * lane; c0 < ld; c0 += 64) {
      float v[2];
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const int c = c0 + u;
        v[u] = 0.0f;
        if (c < nin) {
          const float f = feature(c, n3, deps + r * 6, theta[r], a, ap);
          v[u] = (f - mean[c]) * inv[c];
        }
      }
      xr[c0 >> 1] = __floats2bfloat162_rn(v[0], v[1]);
    }
  }
}

__global__ void k_targets(int64_t n, int n3, int sw, const double *sin, const double *sout,
                          float *tgt) {
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n * n3;
       i += int64_t(gridDim.x) * blockDim.x) {
    const int64_t r = i / n3;
    const int j = int(i - r * n3);
    tgt[i] = float(sout[r * sw + 8 + j] - sin[r * sw + 8 + j]);
  }
}

// partial column sums (sum, sum of squares) over a slab of rows; 32 columns
// per block in x, 8 row lanes in y; FP64 accumulation
__global__ void k_colstats(int64_t n, int cols, const float *x, double *acc) {
  __shared__ double s1[8][32], s2[8][32];
  const int c = blockIdx.x * 32 + threadIdx.x;
  double a = 0.0, b = 0.0;
  if (c < cols) {
    for (int64_t r = blockIdx.y * 8 + threadIdx.y; r < n; r += int64_t(gridDim.y) * 8) {
      const double v = x[r * cols + c];
      a += v;
      b += v * v;
    }
  }
  s1[threadIdx.y][threadIdx.x] = a;
  s2[threadIdx.y][threadIdx.x] = b;
  __syncthreads();
  if (threadIdx.y == 0 && c < cols) {
    for (int k = 1; k < 8; ++k) {
      a += s1[k][threadIdx.x];
      b += s2[k][threadIdx.x];
    }
    atomicAdd(&acc[2 * c], a);
    atomicAdd(&acc[2 * c + 1], b);
  }
}

__global__ void k_colstats_final(int64_t n, int cols, const double *acc, float *mean, float *inv,
                                 float *stdv) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= cols) return;
  const double mu = acc[2 * c] / double(n);
  double var = acc[2 * c + 1] / double(n) - mu * mu;
  if (var < 0.0) var = 0.0;
  const double sd = sqrt(var);
  // spread below 1e-9 of the column's scale: treat the column as constant
  const bool flat = !(sd > 1e-9 * fabs(mu)) || sd == 0.0;
  mean[c] = float(mu);
  if (inv) inv[c] = flat ? 0.0f : float(1.0 / sd);
  if (stdv) stdv[c] = flat ? 0.0f : float(sd);
}

__global__ void k_norm_x(int64_t n, int nin, int ld, const float *feat, const float *mean,
                         const float *inv, bf16 *x) {
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n * ld;
       i += int64_t(gridDim.x) * blockDim.x) {
    const int64_t r = i / ld;
    const int c = int(i - r * ld);
    x[i] = __float2bfloat16(c < nin ? (feat[r * nin + c] - mean[c]) * inv[c] : 0.0f);
  }
}

__global__ void k_norm_t(int64_t n, int nout, int ld, const float *tgt, const float *mean,
                         const float *inv, float *t) {
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n * ld;
       i += int64_t(gridDim.x) * blockDim.x) {
    const int64_t r = i / ld;
    const int c = int(i - r * ld);
    t[i] = c < nout ? (tgt[r * nout + c] - mean[c]) * inv[c] : 0.0f;
  }
}

// dst[c][r] = src[r][c] for a rows x cols bf16 matrix (32 x 32 tiles)
__global__ void k_transpose(int rows, int cols, const bf16 *src, bf16 *dst) {
  __shared__ bf16 tile[32][33];
  const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
  for (int j = threadIdx.y; j < 32; j += 8) {
    const int r = r0 + j, c = c0 + threadIdx.x;
    if (r < rows && c < cols) tile[j][threadIdx.x] = src[size_t(r) * cols + c];
  }
  __syncthreads();
  for (int j = threadIdx.y; j < 32; j += 8) {
    const int c = c0 + j, r = r0 + threadIdx.x;
    if (r < rows && c < cols) dst[size_t(c) * rows + r] = tile[threadIdx.x][j];
  }
}

// MSE on normalised targets: dY = 2 (y - t) / (n n_out) on valid rows and
// columns, 0 elsewhere; bf16 copy and (through a 32 x 32 shared tile) a
// transposed copy; loss sum.  Block (32, 8) per tile of 32 rows x 32 columns.
__global__ void k_loss(int n, int npad, int nout, int ld, const float *y, const float *t, bf16 *dz,
                       bf16 *dzt, float *loss, float scale) {
  __shared__ bf16 tile[32][33];
  const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
  float part = 0.0f;
  for (int j = threadIdx.y; j < 32; j += 8) {
    const int r = r0 + j, c = c0 + threadIdx.x;
    const size_t i = size_t(r) * ld + c;
    const float d = (r < n && c < nout) ? y[i] - t[i] : 0.0f;
    part += d * d;
    const bf16 g = __float2bfloat16(2.0f * d * scale);
    dz[i] = g;
    tile[j][threadIdx.x] = g;
  }
  __syncthreads();
  for (int j = threadIdx.y; j < 32; j += 8)
    dzt[size_t(c0 + j) * npad + r0 + threadIdx.x] = tile[threadIdx.x][j];
  for (int o = 16; o > 0; o >>= 1) part += __shfl_down_sync(0xffffffffu, part, o);
  if (threadIdx.x == 0 && loss) atomicAdd(loss, part * scale);
}

// db[i] = sum_j dzt[i][j] (one warp per row)
__global__ void k_rowsum(int rows, int cols, const bf16 *dzt, float *db) {
  const int row = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (row >= rows) return;
  float s = 0.0f;
  for (int j = lane; j < cols; j += 32) s += __bfloat162float(dzt[size_t(row) * cols + j]);
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if (lane == 0) db[row] = s;
}

// AMSGrad with bias correction (Reddi, Kale, Kumar 2018; the maximum of the
// second-moment estimates replaces it in the step size)
__global__ void k_amsgrad(int64_t count, float *w, const float *g, float *m, float *v, float *vmax,
                          float lr, float b1, float b2, float eps, float bc1, float bc2) {
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < count;
       i += int64_t(gridDim.x) * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    const float vm = fmaxf(vmax[i], vi);
    m[i] = mi;
    v[i] = vi;
    vmax[i] = vm;
    w[i] -= lr * (mi / bc1) / (sqrtf(vm / bc2) + eps);
  }
}

// optimiser constants of the training step (AMSGrad defaults)
constexpr float kBeta1 = 0.9f, kBeta2 = 0.999f, kEps = 1e-8f;

// One AMSGrad step at iteration step >= 1.  The bias corrections 1 - b^t are
// formed in FP64 from the FP32 betas and rounded once: in FP32, 1 - powf(b2, t)
// for b2 near 1 would lose about 5 of its 24 bits to cancellation.
cudaError_t amsgrad(cudaStream_t s, int64_t n, float *w, const float *g, float *m, float *v, float *vmax,
                    float lr, float b1, float b2, float eps, int64_t step) {
  const float bc1 = float(1.0 - pow(double(b1), double(step)));
  const float bc2 = float(1.0 - pow(double(b2), double(step)));
  k_amsgrad<<<blocks_for(n), 256, 0, s>>>(n, w, g, m, v, vmax, lr, b1, b2, eps, bc1, bc2);
  return cudaGetLastError();
}

// bf16 weights and their transpose from the fp32 master copy
__global__ void k_pack(int rows, int cols, const float *w32, bf16 *w, bf16 *wt) {
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < int64_t(rows) * cols;
       i += int64_t(gridDim.x) * blockDim.x) {
    const int r = int(i / cols), c = int(i - int64_t(r) * cols);
    const bf16 b = __float2bfloat16(w32[i]);
    w[i] = b;
    wt[size_t(c) * rows + r] = b;
  }
}

uint64_t splitmix(uint64_t &s) {
  uint64_t z = (s += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

}  // namespace

struct dmn_mlp_s {
  int K, n3, nin, kin, H, nh, nout_pad, L;
  int64_t bmax;
  std::vector<int> din, dout;
  std::vector<int64_t> ow, ob;
  int64_t nparam;
  float *params, *grads, *m, *v, *vmax;
  std::vector<bf16 *> w, wt;
  float *fmean, *finv, *tmean, *tstd, *tinv;
  bf16 *x, *xt;
  std::vector<bf16 *> z, h, ht, dz, dzt;
  float *y, *t;
  double *acc;
  int *err;
  int step;
};

namespace {
dmn_status fail(dmn_status s, const char *fmt, ...) {
  char msg[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(msg, sizeof(msg), fmt, ap);
  va_end(ap);
  set_error_message(msg);
  return s;
}
dmn_status cuda_fail(cudaError_t e, const char *what) {
  return fail(e == cudaErrorMemoryAllocation ? DMN_ERR_OOM : DMN_ERR_CUDA, "%s: %s", what,
              cudaGetErrorString(e));
}
void free_mlp(dmn_mlp p) {
  if (!p) return;
  void *bufs[] = {p->params, p->grads, p->m, p->v, p->vmax, p->fmean, p->finv, p->tmean, p->tstd,
                  p->tinv, p->x, p->xt, p->y, p->t, p->acc, p->err};
  for (void *b : bufs) cudaFree(b);
  for (auto *b : p->w) cudaFree(b);
  for (auto *b : p->wt) cudaFree(b);
  for (auto *b : p->z) cudaFree(b);
  for (auto *b : p->h) cudaFree(b);
  for (auto *b : p->ht) cudaFree(b);
  for (auto *b : p->dz) cudaFree(b);
  for (auto *b : p->dzt) cudaFree(b);
  delete p;
}
template <typename T>
cudaError_t dalloc(T **p, size_t count) {
  return cudaMalloc(reinterpret_cast<void **>(p), sizeof(T) * (count ? count : 1));
}
cudaError_t pack_all(dmn_mlp p, cudaStream_t s) {
  for (int l = 0; l < p->L; ++l) {
    k_pack<<<blocks_for(int64_t(p->dout[l]) * p->din[l]), 256, 0, s>>>(
        p->dout[l], p->din[l], p->params + p->ow[l], p->w[l], p->wt[l]);
  }
  return cudaGetLastError();
}
// copy a batch into the padded workspace (rows n..npad zeroed)
cudaError_t stage_x(dmn_mlp p, cudaStream_t s, int64_t n, int64_t npad, const void *x) {
  const size_t row = sizeof(bf16) * p->kin;
  cudaError_t e = cudaMemcpyAsync(p->x, x, row * n, cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess && npad > n) e = cudaMemsetAsync(p->x + n * p->kin, 0, row * (npad - n), s);
  return e;
}
// forward pass; train = keep pre-activations and transposed activations
cudaError_t forward(dmn_mlp p, cudaStream_t s, int64_t n, int64_t npad, bool train, float *da,
                    const bf16 *x_in) {
  cudaError_t e = cudaSuccess;
  const bf16 *in = x_in;
  for (int l = 0; l < p->L; ++l) {
    EpiArgs ep;
    memset(&ep, 0, sizeof(ep));
    ep.err = p->err;
    ep.bias = p->params + p->ob[l];
    ep.ldc = p->dout[l];
    ep.ldt = int(npad);
    if (l < p->L - 1) {
      ep.mode = EPI_BIAS_SILU;
      ep.z_out = train ? p->z[l] : nullptr;  // pre-activations only for the backward pass
      ep.h_out = p->h[l];
      ep.t_out = train ? p->ht[l] : nullptr;
    } else {
      ep.mode = EPI_BIAS_F32;
      if (train) {
        ep.f_out = p->y;
      } else {
        ep.f_out = da;
        ep.scale = p->tstd;
        ep.shift = p->tmean;
        ep.m_valid = int(n);
        ep.n_valid = p->n3;
        ep.ld_f = p->n3;
      }
    }
    e = gemm(s, in, p->w[l], int(npad), p->dout[l], p->din[l], ep);
    if (e != cudaSuccess) return e;
    if (l < p->L - 1) in = p->h[l];
  }
  return e;
}
}  // namespace

extern "C" dmn_status dmn_mlp_create(dmn_mlp *out, int32_t K, int32_t hidden, int32_t n_hidden,
                                     int64_t max_batch, uint64_t seed) {
  set_error_message("");
  if (!out) return fail(DMN_ERR_ARG, "dmn_mlp_create: out is NULL");
  *out = nullptr;
  if (K < 1 || K > 9) return fail(DMN_ERR_ARG, "dmn_mlp_create: K=%d outside 1..9", K);
  if (hidden < 128 || hidden % 128 || hidden > 4096)
    return fail(DMN_ERR_ARG, "dmn_mlp_create: hidden=%d not a multiple of 128 in 128..4096", hidden);
  if (n_hidden < 1 || n_hidden > 8) return fail(DMN_ERR_ARG, "dmn_mlp_create: n_hidden=%d", n_hidden);
  if (max_batch < 1 || max_batch > (1 << 22))
    return fail(DMN_ERR_ARG, "dmn_mlp_create: max_batch=%lld", (long long)max_batch);
  cudaError_t e = get_encode();
  if (e != cudaSuccess) return cuda_fail(e, "cuTensorMapEncodeTiled entry point");
  dmn_mlp p = new dmn_mlp_s();
  p->K = K;
  p->n3 = 3 * ((1 << K) - 1);
  p->nin = 8 + p->n3 + kExtraFeatures;
  p->kin = int(rup(p->nin, 128));
  p->H = hidden;
  p->nh = n_hidden;
  p->nout_pad = int(rup(p->n3, 128));
  p->L = n_hidden + 1;
  p->bmax = rup(max_batch, 128);
  p->nparam = 0;
  for (int l = 0; l < p->L; ++l) {
    p->din.push_back(l == 0 ? p->kin : hidden);
    p->dout.push_back(l == p->L - 1 ? p->nout_pad : hidden);
    p->ow.push_back(p->nparam);
    p->nparam += int64_t(p->din[l]) * p->dout[l];
    p->ob.push_back(p->nparam);
    p->nparam += p->dout[l];
  }
  p->step = 0;
  p->params = p->grads = p->m = p->v = p->vmax = nullptr;
  p->fmean = p->finv = p->tmean = p->tstd = p->tinv = nullptr;
  p->x = p->xt = nullptr;
  p->y = p->t = nullptr;
  p->acc = nullptr;
  p->err = nullptr;
  p->w.assign(p->L, nullptr);
  p->wt.assign(p->L, nullptr);
  p->z.assign(p->nh, nullptr);
  p->h.assign(p->nh, nullptr);
  p->ht.assign(p->nh, nullptr);
  p->dz.assign(p->L, nullptr);
  p->dzt.assign(p->L, nullptr);
  const int64_t B = p->bmax;
  bool ok = dalloc(&p->params, p->nparam) == cudaSuccess && dalloc(&p->grads, p->nparam) == cudaSuccess &&
            dalloc(&p->m, p->nparam) == cudaSuccess && dalloc(&p->v, p->nparam) == cudaSuccess &&
            dalloc(&p->vmax, p->nparam) == cudaSuccess && dalloc(&p->fmean, p->kin) == cudaSuccess &&
            dalloc(&p->finv, p->kin) == cudaSuccess && dalloc(&p->tmean, p->nout_pad) == cudaSuccess &&
            dalloc(&p->tstd, p->nout_pad) == cudaSuccess && dalloc(&p->tinv, p->nout_pad) == cudaSuccess &&
            dalloc(&p->x, B * p->kin) == cudaSuccess && dalloc(&p->xt, B * p->kin) == cudaSuccess &&
            dalloc(&p->y, B * p->nout_pad) == cudaSuccess && dalloc(&p->t, B * p->nout_pad) == cudaSuccess &&
            dalloc(&p->acc, 2 * int64_t(p->kin > p->nout_pad ? p->kin : p->nout_pad)) == cudaSuccess &&
            dalloc(&p->err, 1) == cudaSuccess;
  for (int l = 0; ok && l < p->L; ++l)
    ok = dalloc(&p->w[l], int64_t(p->din[l]) * p->dout[l]) == cudaSuccess &&
         dalloc(&p->wt[l], int64_t(p->din[l]) * p->dout[l]) == cudaSuccess &&
         dalloc(&p->dz[l], B * p->dout[l]) == cudaSuccess && dalloc(&p->dzt[l], B * p->dout[l]) == cudaSuccess;
  for (int l = 0; ok && l < p->nh; ++l)
    ok = dalloc(&p->z[l], B * hidden) == cudaSuccess && dalloc(&p->h[l], B * hidden) == cudaSuccess &&
         dalloc(&p->ht[l], B * hidden) == cudaSuccess;
  if (!ok) {
    free_mlp(p);
    return fail(DMN_ERR_OOM, "dmn_mlp_create: device allocation failed");
  }
  // seeded initialisation on the host
  std::vector<float> hp(p->nparam, 0.0f);
  uint64_t st = seed * 0x2545F4914F6CDD1Dull + 0x1234567ull;
  for (int l = 0; l < p->L; ++l) {
    const int fan_in = l == 0 ? p->nin : hidden;
    const int rows = l == p->L - 1 ? p->n3 : hidden;
    const float a = 1.0f / sqrtf(float(fan_in));
    for (int r = 0; r < rows; ++r)
      for (int c = 0; c < fan_in; ++c) {
        const double u = double(splitmix(st) >> 11) * (1.0 / 9007199254740992.0);
        hp[p->ow[l] + int64_t(r) * p->din[l] + c] = float((2.0 * u - 1.0) * a);
      }
  }
  const int cmax = p->kin > p->nout_pad ? p->kin : p->nout_pad;
  std::vector<float> ones(cmax, 1.0f);
  if ((e = cudaMemcpy(p->params, hp.data(), sizeof(float) * p->nparam, cudaMemcpyHostToDevice)) != cudaSuccess ||
      (e = cudaMemset(p->m, 0, sizeof(float) * p->nparam)) != cudaSuccess ||
      (e = cudaMemset(p->v, 0, sizeof(float) * p->nparam)) != cudaSuccess ||
      (e = cudaMemset(p->vmax, 0, sizeof(float) * p->nparam)) != cudaSuccess ||
      (e = cudaMemset(p->grads, 0, sizeof(float) * p->nparam)) != cudaSuccess ||
      (e = cudaMemset(p->fmean, 0, sizeof(float) * p->kin)) != cudaSuccess ||
      (e = cudaMemcpy(p->finv, ones.data(), sizeof(float) * p->kin, cudaMemcpyHostToDevice)) != cudaSuccess ||
      (e = cudaMemset(p->tmean, 0, sizeof(float) * p->nout_pad)) != cudaSuccess ||
      (e = cudaMemcpy(p->tstd, ones.data(), sizeof(float) * p->nout_pad, cudaMemcpyHostToDevice)) != cudaSuccess ||
      (e = cudaMemcpy(p->tinv, ones.data(), sizeof(float) * p->nout_pad, cudaMemcpyHostToDevice)) != cudaSuccess ||
      (e = cudaMemset(p->err, 0, sizeof(int))) != cudaSuccess || (e = pack_all(p, 0)) != cudaSuccess ||
      (e = cudaDeviceSynchronize()) != cudaSuccess) {
    free_mlp(p);
    return cuda_fail(e, "dmn_mlp_create");
  }
  *out = p;
  return DMN_OK;
}

extern "C" dmn_status dmn_mlp_destroy(dmn_mlp m) {
  set_error_message("");
  if (!m) return fail(DMN_ERR_ARG, "dmn_mlp_destroy: NULL");
  free_mlp(m);
  return DMN_OK;
}

extern "C" dmn_status dmn_mlp_dims(dmn_mlp m, int32_t *n_in, int32_t *n_in_pad, int32_t *n_out,
                                   int32_t *n_out_pad) {
  if (!m) return fail(DMN_ERR_ARG, "dmn_mlp_dims: NULL");
  if (n_in) *n_in = m->nin;
  if (n_in_pad) *n_in_pad = m->kin;
  if (n_out) *n_out = m->n3;
  if (n_out_pad) *n_out_pad = m->nout_pad;
  return DMN_OK;
}

extern "C" dmn_status dmn_mlp_features(dmn_mlp m, dmn_stream stream, int64_t n, const double *d_deps,
                                       const double *d_theta, const double *d_state_in,
                                       const double *d_state_prev, int64_t state_words,
                                       float *d_feat) {
  set_error_message("");
  if (!m || n < 0 || !d_deps || !d_theta || !d_state_in || !d_feat || state_words < 8 + m->n3)
    return fail(DMN_ERR_ARG, "dmn_mlp_features: invalid argument");
  if (n == 0) return DMN_OK;
  k_features<<<blocks_for(n * m->nin), 256, 0, (cudaStream_t)stream>>>(
      n, m->n3, int(state_words), d_deps, d_theta, d_state_in, d_state_prev, d_feat);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? DMN_OK : cuda_fail(e, "dmn_mlp_features");
}

extern "C" dmn_status dmn_mlp_input(dmn_mlp m, dmn_stream stream, int64_t n, const double *d_deps,
                                    const double *d_theta, const double *d_state_in,
                                    const double *d_state_prev, int64_t state_words,
                                    void *d_x_bf16) {
  set_error_message("");
  if (!m || n < 0 || !d_deps || !d_theta || !d_state_in || !d_x_bf16 || state_words < 8 + m->n3)
    return fail(DMN_ERR_ARG, "dmn_mlp_input: invalid argument");
  if (n == 0) return DMN_OK;
  k_features_norm<<<blocks_for(n * 32), 256, 0, (cudaStream_t)stream>>>(
      n, m->n3, int(state_words), m->kin, d_deps, d_theta, d_state_in, d_state_prev, m->fmean,
      m->finv, static_cast<bf16 *>(d_x_bf16));
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? DMN_OK : cuda_fail(e, "dmn_mlp_input");
}

extern "C" dmn_status dmn_mlp_targets(dmn_mlp m, dmn_stream stream, int64_t n,
                                      const double *d_state_in, const double *d_state_out,
                                      int64_t state_words, float *d_tgt) {
  set_error_message("");
  if (!m || n < 0 || !d_state_in || !d_state_out || !d_tgt || state_words < 8 + m->n3)
    return fail(DMN_ERR_ARG, "dmn_mlp_targets: invalid argument");
  if (n == 0) return DMN_OK;
  k_targets<<<blocks_for(n * m->n3), 256, 0, (cudaStream_t)stream>>>(
      n, m->n3, int(state_words), d_state_in, d_state_out, d_tgt);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? DMN_OK : cuda_fail(e, "dmn_mlp_targets");
}

extern "C" dmn_status dmn_mlp_fit_normalization(dmn_mlp m, dmn_stream stream, int64_t n,
                                                const float *d_feat, const float *d_tgt) {
  set_error_message("");
  if (!m || n < 2 || !d_feat || !d_tgt) return fail(DMN_ERR_ARG, "dmn_mlp_fit_normalization: invalid argument");
  cudaStream_t s = (cudaStream_t)stream;
  const int cmax = m->kin > m->nout_pad ? m->kin : m->nout_pad;
  cudaError_t e = cudaMemsetAsync(m->acc, 0, sizeof(double) * 2 * cmax, s);
  if (e != cudaSuccess) return cuda_fail(e, "memset");
  const unsigned gy = unsigned(n / 8 < 256 ? (n / 8 > 0 ? n / 8 : 1) : 256);
  k_colstats<<<dim3((m->nin + 31) / 32, gy), dim3(32, 8), 0, s>>>(n, m->nin, d_feat, m->acc);
  k_colstats_final<<<(m->nin + 127) / 128, 128, 0, s>>>(n, m->nin, m->acc, m->fmean, m->finv, nullptr);
  e = cudaMemsetAsync(m->acc, 0, sizeof(double) * 2 * cmax, s);
  if (e != cudaSuccess) return cuda_fail(e, "memset");
  k_colstats<<<dim3((m->n3 + 31) / 32, gy), dim3(32, 8), 0, s>>>(n, m->n3, d_tgt, m->acc);
  k_colstats_final<<<(m->n3 + 127) / 128, 128, 0, s>>>(n, m->n3, m->acc, m->tmean, m->tinv, m->tstd);
  e = cudaGetLastError();
  return e == cudaSuccess ? DMN_OK : cuda_fail(e, "dmn_mlp_fit_normalization");
}

extern "C" dmn_status dmn_mlp_normalize_features(dmn_mlp m, dmn_stream stream, int64_t n,
                                                 const float *d_feat, void *d_x_bf16) {
  set_error_message("");
  if (!m || n < 0 || !d_feat || !d_x_bf16) return fail(DMN_ERR_ARG, "dmn_mlp_normalize_features: invalid argument");
  if (n == 0) return DMN_OK;
  k_norm_x<<<blocks_for(n * m->kin), 256, 0, (cudaStream_t)stream>>>(
      n, m->nin, m->kin, d_feat, m->fmean, m->finv, static_cast<bf16 *>(d_x_bf16));
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? DMN_OK : cuda_fail(e, "dmn_mlp_normalize_features");
}

extern "C" dmn_status dmn_mlp_normalize_targets(dmn_mlp m, dmn_stream stream, int64_t n,
                                                const float *d_tgt, float *d_t) {
  set_error_message("");
  if (!m || n < 0 || !d_tgt || !d_t) return fail(DMN_ERR_ARG, "dmn_mlp_normalize_targets: invalid argument");
  if (n == 0) return DMN_OK;
  k_norm_t<<<blocks_for(n * m->nout_pad), 256, 0, (cudaStream_t)stream>>>(
      n, m->n3, m->nout_pad, d_tgt, m->tmean, m->tinv, d_t);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? DMN_OK : cuda_fail(e, "dmn_mlp_normalize_targets");
}

extern "C" dmn_status dmn_mlp_train_step(dmn_mlp m, dmn_stream stream, int64_t n,
                                         const void *d_x_bf16, const float *d_t, float lr,
                                         float *d_loss) {
  set_error_message("");
  if (!m || n < 1 || n > m->bmax || !d_x_bf16 || !d_t || !(lr >= 0.0f))
    return fail(DMN_ERR_ARG, "dmn_mlp_train_step: invalid argument");
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t npad = rup(n, 128);
  cudaError_t e = stage_x(m, s, n, npad, d_x_bf16);
  if (e == cudaSuccess) e = cudaMemcpyAsync(m->t, d_t, sizeof(float) * m->nout_pad * n, cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess && d_loss) e = cudaMemsetAsync(d_loss, 0, sizeof(float), s);
  if (e != cudaSuccess) return cuda_fail(e, "dmn_mlp_train_step staging");
  k_transpose<<<dim3((m->kin + 31) / 32, unsigned((npad + 31) / 32)), dim3(32, 8), 0, s>>>(
      int(npad), m->kin, m->x, m->xt);
  if ((e = forward(m, s, n, npad, true, nullptr, m->x)) != cudaSuccess) return cuda_fail(e, "forward");
  const int Lo = m->L - 1;
  k_loss<<<dim3(m->nout_pad / 32, unsigned(npad / 32)), dim3(32, 8), 0, s>>>(
      int(n), int(npad), m->n3, m->nout_pad, m->y, m->t, m->dz[Lo], m->dzt[Lo], d_loss,
      1.0f / (float(n) * float(m->n3)));
  for (int l = Lo; l >= 0; --l) {
    // weight gradient dW_l = dZ_l^T . input_l  (reduction over the batch)
    EpiArgs ep;
    memset(&ep, 0, sizeof(ep));
    ep.err = m->err;
    ep.mode = EPI_F32;
    ep.f_out = m->grads + m->ow[l];
    ep.ldc = m->din[l];
    const bf16 *inT = l == 0 ? m->xt : m->ht[l - 1];
    if ((e = gemm(s, m->dzt[l], inT, m->dout[l], m->din[l], int(npad), ep)) != cudaSuccess)
      return cuda_fail(e, "wgrad");
    k_rowsum<<<(m->dout[l] + 7) / 8, 256, 0, s>>>(m->dout[l], int(npad), m->dzt[l], m->grads + m->ob[l]);
    if (l > 0) {  // input gradient through W_l and silu' of the layer below
      EpiArgs ed;
      memset(&ed, 0, sizeof(ed));
      ed.err = m->err;
      ed.mode = EPI_DSILU;
      ed.z_in = m->z[l - 1];
      ed.h_out = m->dz[l - 1];
      ed.t_out = m->dzt[l - 1];
      ed.ldc = m->H;
      ed.ldt = int(npad);
      if ((e = gemm(s, m->dz[l], m->wt[l], int(npad), m->din[l], m->dout[l], ed)) != cudaSuccess)
        return cuda_fail(e, "dgrad");
    }
  }
  m->step += 1;
  if ((e = amsgrad(s, m->nparam, m->params, m->grads, m->m, m->v, m->vmax, lr, kBeta1, kBeta2, kEps,
                   m->step)) != cudaSuccess)
    return cuda_fail(e, "amsgrad");
  if ((e = pack_all(m, s)) != cudaSuccess) return cuda_fail(e, "pack");
  return DMN_OK;
}

extern "C" dmn_status dmn_mlp_amsgrad(dmn_stream stream, int64_t n, float *d_w, const float *d_g,
                                      float *d_m, float *d_v, float *d_vmax, float lr, float beta1,
                                      float beta2, float eps, int64_t step) {
  set_error_message("");
  if (n < 0 || step < 1) return fail(DMN_ERR_ARG, "dmn_mlp_amsgrad: n >= 0 and step >= 1 required");
  if (n == 0) return DMN_OK;
  if (!d_w || !d_g || !d_m || !d_v || !d_vmax) return fail(DMN_ERR_ARG, "dmn_mlp_amsgrad: NULL pointer");
  if (!(beta1 >= 0.0f && beta1 < 1.0f) || !(beta2 >= 0.0f && beta2 < 1.0f) || !(eps > 0.0f) ||
      !isfinite(lr))
    return fail(DMN_ERR_ARG, "dmn_mlp_amsgrad: 0 <= beta < 1, eps > 0 required");
  cudaError_t e = amsgrad((cudaStream_t)stream, n, d_w, d_g, d_m, d_v, d_vmax, lr, beta1, beta2, eps, step);
  return e == cudaSuccess ? DMN_OK : cuda_fail(e, "dmn_mlp_amsgrad");
}

extern "C" dmn_status dmn_mlp_get_moments(dmn_mlp m, float *h_m, float *h_v, float *h_vmax) {
  if (!m) return fail(DMN_ERR_ARG, "dmn_mlp_get_moments: NULL");
  cudaError_t e = cudaSuccess;
  if (h_m && e == cudaSuccess) e = cudaMemcpy(h_m, m->m, sizeof(float) * m->nparam, cudaMemcpyDeviceToHost);
  if (h_v && e == cudaSuccess) e = cudaMemcpy(h_v, m->v, sizeof(float) * m->nparam, cudaMemcpyDeviceToHost);
  if (h_vmax && e == cudaSuccess)
    e = cudaMemcpy(h_vmax, m->vmax, sizeof(float) * m->nparam, cudaMemcpyDeviceToHost);
  return e == cudaSuccess ? DMN_OK : cuda_fail(e, "dmn_mlp_get_moments");
}

extern "C" dmn_status dmn_mlp_predict(dmn_mlp m, dmn_stream stream, int64_t n, const void *d_x_bf16,
                                      float *d_da) {
  set_error_message("");
  if (!m || n < 0 || n > m->bmax || !d_x_bf16 || !d_da) return fail(DMN_ERR_ARG, "dmn_mlp_predict: invalid argument");
  if (n == 0) return DMN_OK;
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t npad = rup(n, 128);
  cudaError_t e = cudaSuccess;
  const bf16 *xin = static_cast<const bf16 *>(d_x_bf16);
  if (npad != n || (reinterpret_cast<uintptr_t>(d_x_bf16) & 15)) {  // pad into the workspace
    e = stage_x(m, s, n, npad, d_x_bf16);
    xin = m->x;
  }
  if (e == cudaSuccess) e = forward(m, s, n, npad, false, d_da, xin);
  return e == cudaSuccess ? DMN_OK : cuda_fail(e, "dmn_mlp_predict");
}

extern "C" int64_t dmn_mlp_param_count(dmn_mlp m) { return m ? m->nparam : -1; }

extern "C" dmn_status dmn_mlp_get_params(dmn_mlp m, float *h) {
  if (!m || !h) return fail(DMN_ERR_ARG, "dmn_mlp_get_params: invalid argument");
  cudaError_t e = cudaMemcpy(h, m->params, sizeof(float) * m->nparam, cudaMemcpyDeviceToHost);
  return e == cudaSuccess ? DMN_OK : cuda_fail(e, "dmn_mlp_get_params");
}

extern "C" dmn_status dmn_mlp_set_params(dmn_mlp m, const float *h) {
  if (!m || !h) return fail(DMN_ERR_ARG, "dmn_mlp_set_params: invalid argument");
  cudaError_t e = cudaMemcpy(m->params, h, sizeof(float) * m->nparam, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = pack_all(m, 0);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  return e == cudaSuccess ? DMN_OK : cuda_fail(e, "dmn_mlp_set_params");
}

extern "C" dmn_status dmn_mlp_get_grads(dmn_mlp m, float *h) {
  if (!m || !h) return fail(DMN_ERR_ARG, "dmn_mlp_get_grads: invalid argument");
  cudaError_t e = cudaMemcpy(h, m->grads, sizeof(float) * m->nparam, cudaMemcpyDeviceToHost);
  return e == cudaSuccess ? DMN_OK : cuda_fail(e, "dmn_mlp_get_grads");
}

extern "C" dmn_status dmn_mlp_get_normalization(dmn_mlp m, float *fmean, float *finv, float *tmean,
                                                float *tstd) {
  if (!m) return fail(DMN_ERR_ARG, "dmn_mlp_get_normalization: NULL");
  cudaError_t e = cudaSuccess;
  if (fmean && e == cudaSuccess) e = cudaMemcpy(fmean, m->fmean, sizeof(float) * m->nin, cudaMemcpyDeviceToHost);
  if (finv && e == cudaSuccess) e = cudaMemcpy(finv, m->finv, sizeof(float) * m->nin, cudaMemcpyDeviceToHost);
  if (tmean && e == cudaSuccess) e = cudaMemcpy(tmean, m->tmean, sizeof(float) * m->n3, cudaMemcpyDeviceToHost);
  if (tstd && e == cudaSuccess) e = cudaMemcpy(tstd, m->tstd, sizeof(float) * m->n3, cudaMemcpyDeviceToHost);
  return e == cudaSuccess ? DMN_OK : cuda_fail(e, "dmn_mlp_get_normalization");
}

extern "C" dmn_status dmn_gemm_bf16_tn(dmn_stream stream, int32_t M, int32_t N, int32_t K,
                                       const void *d_a, const void *d_b, float *d_c) {
  set_error_message("");
  if (!d_a || !d_b || !d_c || M <= 0 || N <= 0 || K <= 0 || M % 128 || N % 128 || K % 64)
    return fail(DMN_ERR_ARG, "dmn_gemm_bf16_tn: M, N must be multiples of 128 and K of 64");
  EpiArgs ep;
  memset(&ep, 0, sizeof(ep));
  ep.mode = EPI_F32;
  ep.f_out = d_c;
  ep.ldc = N;
  cudaError_t e = gemm((cudaStream_t)stream, d_a, d_b, M, N, K, ep);
  return e == cudaSuccess ? DMN_OK : cuda_fail(e, "dmn_gemm_bf16_tn");
}
