// mlp_gemm.cuh -- BF16 tensor-core GEMM for the warm-start MLP on sm_103a:
//   C[M x N] = A[M x K] . B[N x K]^T   (A, B bf16 with K contiguous; FP32
//   accumulation in tensor memory), followed by a fused epilogue.
//
// Two forms.  The persistent wide form (below, gemm_bf16_tn_wide) serves N a
// multiple of 256; the tile form serves every other shape (N a multiple of
// 128).  Tile form: one CTA of 128 threads computes a 128 x 128 tile (grid:
// column tiles fastest); two CTAs share an SM, so one's epilogue overlaps the
// other's MMAs:
//   warp 0, lane 0  loads A and B tiles (64 wide in K) with TMA bulk tensor
//                   copies into a 3-stage ring of 128-byte-swizzled shared
//                   memory, signalled by mbarriers with transaction counts;
//   warp 1          allocates 128 TMEM columns; its lane 0 issues
//                   tcgen05.mma (kind::f16, BF16 x BF16 -> F32, M=128,
//                   N=128, K=16 per instruction) and releases each stage with
//                   tcgen05.commit on that stage's "empty" mbarrier;
//   all 4 warps     wait for the final commit, read the accumulator with
//                   tcgen05.ld (warp w owns TMEM lanes 32w..32w+31 = tile rows)
//                   and run the epilogue.  The de-normalised FP32 prediction
//                   (rows of an odd length) goes through the then idle
//                   operand ring: each warp stages its 32 rows and writes
//                   them row by row, the lanes on consecutive columns.
// Every wait is bounded (about two seconds of SM clock): on a timeout the CTA
// records an error code, stops issuing work, frees its TMEM and returns.
#pragma once
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace dmn {
namespace mlp {

constexpr int BM = 128, BN = 128, BK = 64, STAGES = 3;
constexpr int TILE_A = BM * BK * 2, TILE_B = BN * BK * 2;  // bytes per stage
constexpr int GEMM_SMEM = STAGES * (TILE_A + TILE_B) + 1024 + 256;
static_assert(BM * (BN + 1) * 4 <= STAGES * (TILE_A + TILE_B), "staged FP32 tile fits the ring");
constexpr long long kWaitCycles = 4000000000ll;  // ~2 s at 2 GHz

enum Epi {
  EPI_BIAS_SILU = 0,  // z = acc + bias -> Z (bf16), H = silu(z) (bf16), H^T (bf16, optional)
  EPI_BIAS_F32 = 1,   // y = acc + bias -> fp32; optional y * scale + shift on valid rows/cols
  EPI_DSILU = 2,      // dz = acc * silu'(z_in) -> dZ (bf16), dZ^T (bf16)
  EPI_F32 = 3         // plain fp32 store
};

struct EpiArgs {
  int mode;
  int ldc;                     // leading dimension of row-major outputs (= N)
  int ldt;                     // leading dimension of transposed outputs (= M)
  const float *bias;           // [N]
  __nv_bfloat16 *z_out;        // [M x ldc]
  __nv_bfloat16 *h_out;        // [M x ldc]
  __nv_bfloat16 *t_out;        // [N x ldt] transposed copy of h_out / dz
  const __nv_bfloat16 *z_in;   // [M x ldc] pre-activation for silu'
  float *f_out;                // [M x ldc] fp32 output
  const float *scale, *shift;  // [N] de-normalisation (EPI_BIAS_F32, optional)
  int m_valid, n_valid;        // rows / cols written to f_out when scale is set
  int ld_f;                    // leading dimension of f_out
  int *err;                    // error code (0 = fine)
};

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// bounded wait on an mbarrier phase
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity) {
  const long long t0 = clock64();
  while (!mbar_try(bar, parity))
    if (clock64() - t0 > kWaitCycles) return false;
  return true;
}
__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, uint64_t *bar,
                                            int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%3, %4}], [%2];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(x), "r"(y)
      : "memory");
}
// shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups
// 1024 bytes apart (tcgen05 descriptor version 1)
__device__ __forceinline__ uint64_t sdesc_sw128(const void *tile) {
  const uint64_t a = smem_u32(tile);
  return ((a & 0x3FFFFull) >> 4) | (1ull << 16) | (uint64_t(1024 >> 4) << 32) | (1ull << 46) |
         (2ull << 61);
}
// instruction descriptor: D f32, A and B bf16, both K-major, N and M
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | (uint32_t(N >> 3) << 17) | (uint32_t(M >> 4) << 24);
}
__device__ __forceinline__ void umma(uint32_t tmem, uint64_t ad, uint64_t bd, uint32_t idesc,
                                     uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
      "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
}
__device__ __forceinline__ void umma_commit(uint64_t *bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float v[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,"
      "%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// the logistic function; the quotient with the fast reciprocal (a few FP32
// ulp), which the bf16 rounding of every result that uses it hides
__device__ __forceinline__ float sigmoidf_(float z) { return __fdividef(1.0f, 1.0f + __expf(-z)); }

// two 16-column accumulator loads in flight, one wait
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float v[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,"
      "%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,"
      "%15}, [%16];"
      : "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]),
        "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]),
        "=r"(r[30]), "=r"(r[31])
      : "r"(taddr + 16u));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// The epilogue of 16 accumulator columns n..n+15 of output row r, every mode
// but the staged de-normalised prediction (EPI_BIAS_F32 with scale)
__device__ __forceinline__ void epi_chunk16(const EpiArgs &ep, int r, int n, const float v[16]) {
  if (ep.mode == EPI_BIAS_SILU) {
    __align__(16) __nv_bfloat16 zb[16], hb[16];
    __align__(16) float bb[16];  // the chunk's biases, four vector loads (n is a multiple of 16)
#pragma unroll
    for (int q = 0; q < 4; ++q) reinterpret_cast<float4 *>(bb)[q] = reinterpret_cast<const float4 *>(ep.bias + n)[q];
#pragma unroll
    for (int i = 0; i < 16; ++i) {
      const float z = v[i] + bb[i];
      zb[i] = __float2bfloat16(z);
      hb[i] = __float2bfloat16(z * sigmoidf_(z));
    }
    if (ep.z_out) {
      uint4 *zo = reinterpret_cast<uint4 *>(ep.z_out + size_t(r) * ep.ldc + n);
      zo[0] = reinterpret_cast<uint4 *>(zb)[0];
      zo[1] = reinterpret_cast<uint4 *>(zb)[1];
    }
    uint4 *ho = reinterpret_cast<uint4 *>(ep.h_out + size_t(r) * ep.ldc + n);
    ho[0] = reinterpret_cast<uint4 *>(hb)[0];
    ho[1] = reinterpret_cast<uint4 *>(hb)[1];
    if (ep.t_out) {
#pragma unroll
      for (int i = 0; i < 16; ++i) ep.t_out[size_t(n + i) * ep.ldt + r] = hb[i];
    }
  } else if (ep.mode == EPI_DSILU) {
    __align__(16) __nv_bfloat16 db[16];
    const __nv_bfloat16 *zi = ep.z_in + size_t(r) * ep.ldc + n;
#pragma unroll
    for (int i = 0; i < 16; ++i) {
      const float z = __bfloat162float(zi[i]);
      const float sg = sigmoidf_(z);
      db[i] = __float2bfloat16(v[i] * sg * (1.0f + z * (1.0f - sg)));
    }
    uint4 *dout = reinterpret_cast<uint4 *>(ep.h_out + size_t(r) * ep.ldc + n);
    dout[0] = reinterpret_cast<uint4 *>(db)[0];
    dout[1] = reinterpret_cast<uint4 *>(db)[1];
    if (ep.t_out) {
#pragma unroll
      for (int i = 0; i < 16; ++i) ep.t_out[size_t(n + i) * ep.ldt + r] = db[i];
    }
  } else if (ep.mode == EPI_BIAS_F32) {
    float4 *fo = reinterpret_cast<float4 *>(ep.f_out + size_t(r) * ep.ldc + n);
#pragma unroll
    for (int q = 0; q < 4; ++q)
      fo[q] = make_float4(v[4 * q] + ep.bias[n + 4 * q], v[4 * q + 1] + ep.bias[n + 4 * q + 1],
                          v[4 * q + 2] + ep.bias[n + 4 * q + 2], v[4 * q + 3] + ep.bias[n + 4 * q + 3]);
  } else {  // EPI_F32
    float4 *fo = reinterpret_cast<float4 *>(ep.f_out + size_t(r) * ep.ldc + n);
#pragma unroll
    for (int q = 0; q < 4; ++q) fo[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
  }
}

__global__ void __launch_bounds__(128, 2)
    gemm_bf16_tn(const __grid_constant__ CUtensorMap map_a, const __grid_constant__ CUtensorMap map_b,
                 int K, const EpiArgs ep) {
  extern __shared__ __align__(1024) unsigned char gsm[];
  unsigned char *base = reinterpret_cast<unsigned char *>(
      (reinterpret_cast<uintptr_t>(gsm) + 1023) & ~uintptr_t(1023));
  unsigned char *sa = base;                         // STAGES x TILE_A
  unsigned char *sb = base + STAGES * TILE_A;       // STAGES x TILE_B
  uint64_t *full = reinterpret_cast<uint64_t *>(sb + STAGES * TILE_B);
  uint64_t *empty = full + STAGES;
  uint64_t *done = empty + STAGES;
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(done + 1);
  int *fail = reinterpret_cast<int *>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // column tiles fastest: the CTAs that share an A panel run together and
  // read it from L2 (the A panel of a 65,536-row batch is larger than L2)
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  const int nk = K / BK;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(done, 1);
    *fail = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(128u));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;

  if (warp == 0 && lane == 0) {  // ---- TMA producer ----
    for (int kb = 0; kb < nk; ++kb) {
      const int s = kb % STAGES;
      if (kb >= STAGES && !mbar_wait(&empty[s], ((kb / STAGES) - 1) & 1)) {
        atomicExch(fail, 1);
        break;
      }
      if (*(volatile int *)fail) break;
      mbar_expect_tx(&full[s], TILE_A + TILE_B);
      tma_load_2d(sa + s * TILE_A, &map_a, &full[s], kb * BK, m0);
      tma_load_2d(sb + s * TILE_B, &map_b, &full[s], kb * BK, n0);
    }
  } else if (warp == 1 && lane == 0) {  // ---- MMA issuer ----
    const uint32_t idesc = idesc_bf16(BM, BN);
    int kb = 0;
    for (; kb < nk; ++kb) {
      const int s = kb % STAGES;
      if (!mbar_wait(&full[s], (kb / STAGES) & 1)) {
        atomicExch(fail, 1);
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint64_t ad = sdesc_sw128(sa + s * TILE_A), bd = sdesc_sw128(sb + s * TILE_B);
#pragma unroll
      for (int k = 0; k < BK / 16; ++k)  // 16 bf16 = 32 bytes per step inside the swizzle atom
        umma(tmem, ad + 2 * k, bd + 2 * k, idesc, (kb > 0 || k > 0) ? 1u : 0u);
      umma_commit(&empty[s]);
    }
    umma_commit(done);  // arrives once all issued MMAs have completed
  }
  __syncwarp();
  // ---- epilogue: all 4 warps ----
  bool ok = mbar_wait(done, 0);
  // the epilogue's tcgen05.ld is warp-synchronous: decide CTA-wide
  ok = __syncthreads_and(ok && *(volatile int *)fail == 0);
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (!ok) {
    if (threadIdx.x == 0 && ep.err) atomicExch(ep.err, 1);
  } else {
    const int r = m0 + warp * 32 + lane;  // tile row owned by this thread
    const uint32_t trow = tmem + (uint32_t(warp * 32) << 16);
    for (int c0 = 0; c0 < BN; c0 += 16) {
      float v[16];
      tmem_ld16(trow + c0, v);
      const int n = n0 + c0;
      if (ep.mode == EPI_BIAS_F32 && ep.scale) {  // staged: the ring holds no operands once `done` has fired
        float *srow = reinterpret_cast<float *>(base) + (warp * 32 + lane) * (BN + 1);
#pragma unroll
        for (int i = 0; i < 16; ++i) srow[c0 + i] = v[i];
      } else {
        epi_chunk16(ep, r, n, v);
      }
    }
    if (ep.mode == EPI_BIAS_F32 && ep.scale) {
      // de-normalised prediction on valid rows and columns: the warp writes
      // its 32 staged rows, lane l on columns l, l+32, l+64, l+96
      __syncwarp();
      const float *tile = reinterpret_cast<const float *>(base);
      float bb[4], sc[4], sh[4];
      bool cv[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int n = n0 + lane + 32 * q;
        cv[q] = n < ep.n_valid;
        bb[q] = cv[q] ? ep.bias[n] : 0.0f;
        sc[q] = cv[q] ? ep.scale[n] : 0.0f;
        sh[q] = cv[q] ? ep.shift[n] : 0.0f;
      }
      for (int rr = 0; rr < 32; ++rr) {
        const int row = warp * 32 + rr, rg = m0 + row;
        if (rg >= ep.m_valid) break;
        float *dst = ep.f_out + size_t(rg) * ep.ld_f + n0 + lane;
#pragma unroll
        for (int q = 0; q < 4; ++q)
          if (cv[q]) dst[32 * q] = (tile[row * (BN + 1) + lane + 32 * q] + bb[q]) * sc[q] + sh[q];
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 1) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(128u));
  }
}

// ---------------------------------------------------------------- wide form
// Persistent form for N a multiple of 256 (the network's forward layers: N =
// 512 or 768): one CTA per SM loops over 128 x 256 tiles (column tiles
// fastest, so the CTAs sharing an A panel run together and read it from L2).
// Six warps with fixed roles:
//   warp 0, lane 0  TMA producer: A (128 x 64) and B (256 x 64) of each K step
//                   into a 4-stage ring (48 KB per stage);
//   warp 1          allocates all 512 TMEM columns (two 256-column FP32
//                   accumulators); its lane 0 issues tcgen05.mma (M = 128,
//                   N = 256, K = 16) and commits each stage to its "empty"
//                   barrier and each finished tile to its accumulator's
//                   "full" barrier;
//   warps 2..9      the epilogue, two warps per TMEM lane quarter: warp w
//                   reads lanes 32 (w % 4).. (tile rows) of one half of the
//                   columns with tcgen05.ld, applies the fused epilogue and
//                   releases the accumulator ("empty", one arrival per warp),
//                   so the MMAs of the next tile run into the other
//                   accumulator meanwhile.  (One warp per quarter could not
//                   keep up: the SiLU epilogue of a 128 x 256 tile is longer
//                   than its MMAs.)
// The de-normalised FP32 prediction is staged per warp (32 rows x 16 columns)
// and written two rows at a time, the lanes on consecutive columns.  Every
// wait is bounded as in the form above.
constexpr int WBN = 256, WST = 4, WEPI = 8;  // epilogue warps
constexpr int WTILE_B = WBN * BK * 2;
constexpr int WSTAGE = TILE_A + WTILE_B;  // 48 KB, a multiple of 1024
constexpr int WSTAGE_EPI = WEPI * 32 * 17 * 4;  // staging of the prediction: per warp 32 x 17 floats
constexpr int WGEMM_SMEM = WST * WSTAGE + WSTAGE_EPI + 1024 + 256;
static_assert(WGEMM_SMEM <= 232448, "opt-in shared memory per CTA");

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__global__ void __launch_bounds__(64 + 32 * WEPI, 1)
    gemm_bf16_tn_wide(const __grid_constant__ CUtensorMap map_a, const __grid_constant__ CUtensorMap map_b,
                      int M, int N, int K, const EpiArgs ep) {
  extern __shared__ __align__(1024) unsigned char gsm[];
  unsigned char *base = reinterpret_cast<unsigned char *>(
      (reinterpret_cast<uintptr_t>(gsm) + 1023) & ~uintptr_t(1023));
  float *stage_epi = reinterpret_cast<float *>(base + WST * WSTAGE);
  uint64_t *full = reinterpret_cast<uint64_t *>(base + WST * WSTAGE + WSTAGE_EPI);
  uint64_t *empty = full + WST;
  uint64_t *accf = empty + WST;  // 2: accumulator full (MMA -> epilogue)
  uint64_t *acce = accf + 2;     // 2: accumulator empty (epilogue -> MMA)
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(acce + 2);
  int *fail = reinterpret_cast<int *>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ntn = N / WBN, ntiles = (M / BM) * ntn, nk = K / BK;

  if (threadIdx.x == 0) {
    for (int st = 0; st < WST; ++st) {
      mbar_init(&full[st], 1);
      mbar_init(&empty[st], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&accf[b], 1);
      mbar_init(&acce[b], WEPI);
    }
    *fail = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(512u));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {  // ---- TMA producer ----
      int it = 0;
      for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int m0 = (t / ntn) * BM, n0 = (t % ntn) * WBN;
        for (int kb = 0; kb < nk; ++kb, ++it) {
          const int st = it % WST;
          if (it >= WST && !mbar_wait(&empty[st], ((it / WST) - 1) & 1)) {
            atomicExch(fail, 1);
            break;
          }
          if (*(volatile int *)fail) break;
          mbar_expect_tx(&full[st], WSTAGE);
          tma_load_2d(base + st * WSTAGE, &map_a, &full[st], kb * BK, m0);
          tma_load_2d(base + st * WSTAGE + TILE_A, &map_b, &full[st], kb * BK, n0);
        }
        if (*(volatile int *)fail) break;
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {  // ---- MMA issuer ----
      const uint32_t idesc = idesc_bf16(BM, WBN);
      int it = 0, j = 0;
      for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++j) {
        const int b = j & 1;
        if (j >= 2 && !mbar_wait(&acce[b], ((j >> 1) - 1) & 1)) {
          atomicExch(fail, 1);
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t acc = tmem + uint32_t(b * WBN);
        bool bad = false;
        for (int kb = 0; kb < nk; ++kb, ++it) {
          const int st = it % WST;
          if (!mbar_wait(&full[st], (it / WST) & 1)) {
            atomicExch(fail, 1);
            bad = true;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint64_t ad = sdesc_sw128(base + st * WSTAGE), bd = sdesc_sw128(base + st * WSTAGE + TILE_A);
#pragma unroll
          for (int k = 0; k < BK / 16; ++k)
            umma(acc, ad + 2 * k, bd + 2 * k, idesc, (kb > 0 || k > 0) ? 1u : 0u);
          umma_commit(&empty[st]);
        }
        if (bad) break;
        umma_commit(&accf[b]);  // arrives once this tile's MMAs have completed
      }
    }
  } else {  // ---- epilogue: warps 2..9 ----
    const int qd = warp & 3;  // TMEM lane quarter = tile rows 32 qd ..
    const int ch0 = ((warp - 2) >> 2) * (WBN / (WEPI / 4));  // this warp's columns
    constexpr int CW = WBN / (WEPI / 4);
    float *stg = stage_epi + (warp - 2) * 32 * 17;
    int j = 0;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++j) {
      const int b = j & 1;
      const bool ok = mbar_wait(&accf[b], (j >> 1) & 1);
      if (!__all_sync(0xffffffffu, ok) || *(volatile int *)fail) {
        if (lane == 0) atomicExch(fail, 1);
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const int m0 = (t / ntn) * BM, n0 = (t % ntn) * WBN;
      const int r = m0 + qd * 32 + lane;
      const uint32_t trow = tmem + (uint32_t(qd * 32) << 16) + uint32_t(b * WBN);
      if (ep.mode == EPI_BIAS_F32 && ep.scale) {
        for (int c0 = ch0; c0 < ch0 + CW; c0 += 16) {
          float v[16];
          tmem_ld16(trow + c0, v);
#pragma unroll
          for (int i = 0; i < 16; ++i) stg[lane * 17 + i] = v[i];
          __syncwarp();
          // lanes 0..15 on row rr, 16..31 on row rr + 1, consecutive columns
          const int cl = lane & 15, n = n0 + c0 + cl;
          const bool cv = n < ep.n_valid;
          const float bb = cv ? ep.bias[n] : 0.0f, sc = cv ? ep.scale[n] : 0.0f, sh = cv ? ep.shift[n] : 0.0f;
          for (int rr = lane >> 4; rr < 32; rr += 2) {
            const int rg = m0 + qd * 32 + rr;
            if (cv && rg < ep.m_valid) ep.f_out[size_t(rg) * ep.ld_f + n] = (stg[rr * 17 + cl] + bb) * sc + sh;
          }
          __syncwarp();
        }
      } else {
        for (int c0 = ch0; c0 < ch0 + CW; c0 += 32) {
          float v[32];
          tmem_ld32(trow + c0, v);
          epi_chunk16(ep, r, n0 + c0, v);
          epi_chunk16(ep, r, n0 + c0 + 16, v + 16);
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(&acce[b]);
    }
  }
  __syncwarp();  // lanes 1..31 of the producer and MMA warps wait for lane 0 here
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (threadIdx.x == 0 && *(volatile int *)fail && ep.err) atomicExch(ep.err, 1);
  if (warp == 1) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512u));
  }
}

}  // namespace mlp
}  // namespace dmn
