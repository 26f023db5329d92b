// mlp_tc.cu -- the MLP's products on the 5th-generation tensor cores.
//
// Forward and input gradient: out[M x N] = act(A[M x K] . B[N x K]^T + bias),
// BF16 operands, FP32 accumulation in tensor memory (TMEM), N and K in {64,
// 256}; act 1 applies GELU, act 2 multiplies by GELU'(g) of a stored
// pre-activation g (the input gradient through the activation).  Weight
// gradient: a split-K product D[M x N] = A[M x K] . B[N x K]^T with K the
// batch (gemm_tn_splitk_tc below).  Persistent
// CTAs (one per SM): each loads B once into shared memory and then walks
// 128-row tiles of A.  Per tile: one thread issues K/16 tcgen05.mma (128 x N
// x 16) on the A tile in shared memory and commits them to an mbarrier, all
// threads wait on it (bounded), start copying the next A tile into the now
// free buffer (cp.async), and meanwhile each warp reads its 32 accumulator
// rows from TMEM (tcgen05.ld) and applies bias, GELU and the BF16/FP32
// stores.
//
// Shared-memory operand layout (K-major, no swizzle): 8-row x 16-byte core
// matrices; core matrix (row group g, 16-byte K chunk c) sits at byte
// (g * K/8 + c) * 128, so neighbouring K chunks are 128 bytes apart (the
// descriptor's leading-dimension offset) and neighbouring row groups K/8 *
// 128 bytes apart (its stride-dimension offset).
#include <cuda_bf16.h>

#include <algorithm>

#include "pg_host.h"

namespace pg {

namespace {

constexpr int TM = 128;
constexpr int kTcThreads = 128;
constexpr long long kSpinLimit = 20000000;   // mbarrier polls before giving up

__device__ __forceinline__ uint32_t su32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// GELU in its tanh form, 0.5 x (1 + tanh(sqrt(2/pi) (x + 0.044715 x^3))),
// written as h + h t with h = x / 2 and the tanh argument x (c0 + c1 x^2);
// hardware tanh approximation.  The same expression as mlp.cu and the fused
// forward (mlp_fused.cu).
__device__ __forceinline__ float gelu_tc(float x) {
  const float p = fmaf(x * x, 0.035677408136300125f, 0.7978845608028654f);
  float t;
  asm("tanh.approx.f32 %0, %1;" : "=f"(t) : "f"(x * p));
  const float h = 0.5f * x;
  return fmaf(h, t, h);
}

// Its derivative, as mlp.cu's gelu_grad.
__device__ __forceinline__ float gelu_grad_tc(float x) {
  const float u = 0.7978845608028654f * (x + 0.044715f * x * x * x);
  float t;
  asm("tanh.approx.f32 %0, %1;" : "=f"(t) : "f"(u));
  return 0.5f * (1.0f + t) +
         0.5f * x * (1.0f - t * t) * 0.7978845608028654f * (1.0f + 0.134145f * x * x);
}

// 64-bit shared-memory matrix descriptor: start address, leading and stride
// byte offsets (all >> 4), the fixed 0b001 at bits 46-48, no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((addr & 0x3FFFF) >> 4);
  d |= (uint64_t)((lbo & 0x3FFFF) >> 4) << 16;
  d |= (uint64_t)((sbo & 0x3FFFF) >> 4) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// Instruction descriptor, kind::f16: D FP32, A and B BF16, both K-major.
__host__ __device__ constexpr uint32_t instr_desc(int m, int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) |
         ((uint32_t)(m >> 4) << 24);
}

// 16 FP32 values rounded to BF16 (nearest even, in pairs) and written as two
// 16-byte stores; dst must be 16-byte aligned.
__device__ __forceinline__ void store_bf16x16(__nv_bfloat16 *dst, const float (&v)[16]) {
  uint32_t w[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(v[2 * j], v[2 * j + 1]);
    w[j] = *reinterpret_cast<const uint32_t *>(&h);
  }
  reinterpret_cast<uint4 *>(dst)[0] = make_uint4(w[0], w[1], w[2], w[3]);
  reinterpret_cast<uint4 *>(dst)[1] = make_uint4(w[4], w[5], w[6], w[7]);
}

// copy rows [0, rows) of a K-wide BF16 matrix (row stride ld) into the
// core-matrix layout; rows in [rows, R) are zero-filled
template <int K>
__device__ __forceinline__ void load_tile(uint8_t *dst, const __nv_bfloat16 *src, int ld, int rows,
                                          int R) {
  constexpr int KC = K / 8;   // 16-byte chunks per row
  for (int idx = threadIdx.x; idx < R * KC; idx += kTcThreads) {
    const int r = idx / KC, c = idx - r * KC;
    const uint32_t off = (uint32_t)(((r >> 3) * KC + c) * 128 + (r & 7) * 16);
    const bool ok = r < rows;
    const __nv_bfloat16 *s = src + (size_t)(ok ? r : 0) * ld + c * 8;
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(su32(dst + off)),
                 "l"(s), "r"(ok ? 16 : 0));
  }
}

// Poll the mbarrier for the given phase parity at most kSpinLimit times.
__device__ __forceinline__ bool wait_parity_bounded(uint64_t *mbar, uint32_t phase) {
  uint32_t done = 0;
  long long spins = 0;
  while (!done) {
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(su32(mbar)), "r"(phase));
    if (!done && ++spins > kSpinLimit) break;
  }
  return done != 0;
}

template <int N, int K>
__global__ void __launch_bounds__(kTcThreads, 1)
gemm_tc_kernel(const __nv_bfloat16 *__restrict__ A, int lda, const __nv_bfloat16 *__restrict__ B,
               int ldb, int64_t M, const float *__restrict__ bias, int act, float *out_f32,
               __nv_bfloat16 *out_bf16, __nv_bfloat16 *pre_bf16,
               const __nv_bfloat16 *__restrict__ gin, int ldc, int *err) {
  constexpr int NCOLS = N < 32 ? 32 : N;       // TMEM columns (power of two >= 32)
  constexpr uint32_t SB = N * K * 2, SA = TM * K * 2;
  extern __shared__ __align__(1024) uint8_t smem[];
  uint8_t *sB = smem;
  uint8_t *sA = smem + SB;
  uint64_t *mbar = reinterpret_cast<uint64_t *>(smem + SB + SA);
  uint32_t *tslot = reinterpret_cast<uint32_t *>(smem + SB + SA + 8);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t ntiles = (M + TM - 1) / TM;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                     su32(tslot)), "r"(NCOLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
  }
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(su32(mbar)));
    asm volatile("fence.mbarrier_init.release.cluster;\n");
  }
  load_tile<K>(sB, B, ldb, N, N);
  asm volatile("cp.async.commit_group;\n");
  asm volatile("tcgen05.fence::before_thread_sync;\n");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n");
  const uint32_t tmem = *tslot;
  const uint32_t idesc = instr_desc(TM, N);
  uint32_t phase = 0;
  bool failed = false;

  // The A tile of the next iteration is copied while this tile's epilogue
  // runs: once the MMA has completed (mbarrier), the shared A buffer is free.
  auto copy_a = [&](int64_t t) {
    const int64_t m = t * TM;
    load_tile<K>(sA, A + (size_t)m * lda, lda, (int)((M - m) < TM ? (M - m) : TM), TM);
    asm volatile("cp.async.commit_group;\n");
  };
  if ((int64_t)blockIdx.x < ntiles) copy_a(blockIdx.x);
  for (int64_t tile = blockIdx.x; tile < ntiles && !failed; tile += gridDim.x) {
    const int64_t m0 = tile * TM;
    asm volatile("cp.async.wait_group 0;\n");
    asm volatile("fence.proxy.async.shared::cta;\n");
    __syncthreads();
    if (threadIdx.x == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;\n");
#pragma unroll
      for (int ks = 0; ks < K / 16; ++ks) {
        const uint64_t da = smem_desc(su32(sA) + ks * 256, 128, (K / 8) * 128);
        const uint64_t db = smem_desc(su32(sB) + ks * 256, 128, (K / 8) * 128);
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
            "l"(da), "l"(db), "r"(idesc), "r"(ks));
      }
      asm volatile(
          "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
              su32(mbar)));
    }
    // wait for the accumulator (bounded).  The CTA decides together whether
    // the wait failed, so every thread leaves the loop at the same point and
    // no aligned tcgen05 instruction or barrier is reached by part of it.
    {
      const bool done = wait_parity_bounded(mbar, phase);
      failed = __syncthreads_or(!done) != 0;
      if (failed) {
        if (threadIdx.x == 0) atomicCAS(err, 0, 1);
        // the MMAs may still be running: give them a second bounded wait
        // before the TMEM is released below, and let the copies in flight land
        wait_parity_bounded(mbar, phase);
        asm volatile("cp.async.wait_group 0;\n");
        __syncthreads();
      }
    }
    phase ^= 1u;
    if (failed) break;
    if (tile + gridDim.x < ntiles) copy_a(tile + gridDim.x);
    asm volatile("tcgen05.fence::after_thread_sync;\n");
    const int64_t row = m0 + warp * 32 + lane;
#pragma unroll 1
    for (int c0 = 0; c0 < N; c0 += 16) {
      uint32_t r[16];
      const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
          "%14,%15}, [%16];\n"
          : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
            "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
            "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
          : "r"(taddr));
      asm volatile("tcgen05.wait::ld.sync.aligned;\n");
      if (row < M) {
        // 16 consecutive columns of this thread's row: 16-byte vector loads
        // of the bias and 16-byte stores (32 B of BF16 or 64 B of FP32)
        const size_t o = (size_t)row * ldc + c0;
        float v[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
        if (bias) {
#pragma unroll
          for (int j = 0; j < 16; j += 4) {
            const float4 b4 = *reinterpret_cast<const float4 *>(bias + c0 + j);
            v[j] += b4.x; v[j + 1] += b4.y; v[j + 2] += b4.z; v[j + 3] += b4.w;
          }
        }
        if (pre_bf16) store_bf16x16(pre_bf16 + o, v);
        if (act == 1) {
#pragma unroll
          for (int j = 0; j < 16; ++j) v[j] = gelu_tc(v[j]);
        } else if (act == 2) {
          // times GELU'(g): 16 BF16 pre-activations in two 16-byte loads
          const uint4 g0 = *reinterpret_cast<const uint4 *>(gin + o);
          const uint4 g1 = *reinterpret_cast<const uint4 *>(gin + o + 8);
          const uint32_t gw[8] = {g0.x, g0.y, g0.z, g0.w, g1.x, g1.y, g1.z, g1.w};
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            const __nv_bfloat162 h = *reinterpret_cast<const __nv_bfloat162 *>(&gw[j]);
            v[2 * j] *= gelu_grad_tc(__low2float(h));
            v[2 * j + 1] *= gelu_grad_tc(__high2float(h));
          }
        }
        if (out_f32) {
#pragma unroll
          for (int j = 0; j < 16; j += 4)
            *reinterpret_cast<float4 *>(out_f32 + o + j) = make_float4(v[j], v[j + 1], v[j + 2], v[j + 3]);
        }
        if (out_bf16) store_bf16x16(out_bf16 + o, v);
      }
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n");
    __syncthreads();
  }
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;\n");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem),
                 "r"(NCOLS));
  }
}

template <int N, int K>
cudaError_t launch_tc(const __nv_bfloat16 *A, int lda, const __nv_bfloat16 *B, int ldb, int64_t M,
                      const float *bias, int act, float *out_f32, __nv_bfloat16 *out_bf16,
                      __nv_bfloat16 *pre_bf16, const __nv_bfloat16 *gin, int ldc, cudaStream_t st,
                      int *err) {
  constexpr size_t smem = (size_t)N * K * 2 + (size_t)TM * K * 2 + 16;
  // the attribute belongs to the current device's context: set it on every
  // launch (cheap), so a first launch on another device is configured too
  cudaError_t e = cudaFuncSetAttribute(gemm_tc_kernel<N, K>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t ntiles = (M + TM - 1) / TM;
  const int grid = (int)(ntiles < sms ? ntiles : sms);
  gemm_tc_kernel<N, K><<<grid, kTcThreads, smem, st>>>(A, lda, B, ldb, M, bias, act, out_f32,
                                                       out_bf16, pre_bf16, gin, ldc, err);
  note_launches(1);
  return cudaGetLastError();
}

}  // namespace

// Forward products of the MLP on tcgen05; N and K must be 64 or 256, all row
// strides multiples of 8 elements, bias and outputs 16-byte aligned.  *err (device) is set to 1 if a CTA gave
// up waiting for its accumulator.
cudaError_t gemm_nt_tc(const __nv_bfloat16 *A, int lda, const __nv_bfloat16 *B, int ldb,
                       int64_t M, int N, int K, const float *bias, int act, float *out_f32,
                       __nv_bfloat16 *out_bf16, __nv_bfloat16 *pre_bf16, int ldc, cudaStream_t st,
                       int *err, const __nv_bfloat16 *gin) {
  if (M == 0) return cudaSuccess;
  if (lda % 8 || ldb % 8 || ldc % 8 || !err || (act == 2 && !gin)) return cudaErrorInvalidValue;
  if (((uintptr_t)bias | (uintptr_t)out_f32 | (uintptr_t)out_bf16 | (uintptr_t)pre_bf16 |
       (uintptr_t)gin) % 16)
    return cudaErrorInvalidValue;
  if (N == 256 && K == 256)
    return launch_tc<256, 256>(A, lda, B, ldb, M, bias, act, out_f32, out_bf16, pre_bf16, gin, ldc, st, err);
  if (N == 256 && K == 64)
    return launch_tc<256, 64>(A, lda, B, ldb, M, bias, act, out_f32, out_bf16, pre_bf16, gin, ldc, st, err);
  if (N == 64 && K == 256)
    return launch_tc<64, 256>(A, lda, B, ldb, M, bias, act, out_f32, out_bf16, pre_bf16, gin, ldc, st, err);
  if (N == 64 && K == 64)
    return launch_tc<64, 64>(A, lda, B, ldb, M, bias, act, out_f32, out_bf16, pre_bf16, gin, ldc, st, err);
  return cudaErrorNotSupported;
}

// ------------------------------------------------------ split-K product ---
namespace {

constexpr int KC = 64;           // K elements per pipeline chunk (128 bytes per row)

// copy the K chunk [k0, k0 + KC) of rows [0, rows) of a BF16 matrix (row
// stride ld, K valid columns) into the core-matrix layout; rows >= rows and
// columns >= K are zero-filled
__device__ __forceinline__ void load_chunk(uint8_t *dst, const __nv_bfloat16 *src, int64_t ld,
                                           int rows, int R, int64_t k0, int64_t K) {
  constexpr int CC = KC / 8;   // 16-byte chunks per row
  for (int idx = threadIdx.x; idx < R * CC; idx += kTcThreads) {
    const int r = idx / CC, c = idx - r * CC;
    const uint32_t off = (uint32_t)(((r >> 3) * CC + c) * 128 + (r & 7) * 16);
    const bool ok = r < rows && k0 + c * 8 < K;
    const __nv_bfloat16 *s = src + (ok ? (size_t)r * ld + (size_t)(k0 + c * 8) : 0);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(su32(dst + off)),
                 "l"(s), "r"(ok ? 16 : 0));
  }
}

// CTA (m-tile mt, split s): D_s = A[mt rows, K slice] . B[:, K slice]^T in
// TMEM over chunks [c0, c1) with a two-stage copy pipeline, then the FP32
// partial [128 x N] to part[s][mt * 128 + row][col].
template <int N>
__global__ void __launch_bounds__(kTcThreads, 1)
gemm_splitk_tc_kernel(const __nv_bfloat16 *__restrict__ A, int64_t lda, int Mrows,
                      const __nv_bfloat16 *__restrict__ B, int64_t ldb, int64_t K, int cps,
                      int mtiles, float *part, int *err) {
  constexpr int NCOLS = N < 32 ? 32 : N;
  constexpr uint32_t SA = TM * KC * 2, SB = N * KC * 2;
  extern __shared__ __align__(1024) uint8_t smem[];
  // stage st: A at smem + st * SA, B at smem + 2 SA + st * SB
  auto sA = [&](int st) { return smem + st * SA; };
  auto sB = [&](int st) { return smem + 2 * SA + st * SB; };
  uint64_t *mbar = reinterpret_cast<uint64_t *>(smem + 2 * SA + 2 * SB);
  uint32_t *tslot = reinterpret_cast<uint32_t *>(smem + 2 * SA + 2 * SB + 16);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int mt = blockIdx.x % mtiles, sp = blockIdx.x / mtiles;
  const int64_t nchunks = (K + KC - 1) / KC;
  const int64_t c0 = (int64_t)sp * cps;
  const int64_t c1 = c0 + cps < nchunks ? c0 + cps : nchunks;
  const int rows = Mrows - mt * TM < TM ? Mrows - mt * TM : TM;
  const __nv_bfloat16 *Am = A + (size_t)mt * TM * lda;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                     su32(tslot)), "r"(NCOLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
  }
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(su32(&mbar[0])));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(su32(&mbar[1])));
    asm volatile("fence.mbarrier_init.release.cluster;\n");
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n");
  const uint32_t tmem = *tslot;
  const uint32_t idesc = instr_desc(TM, N);
  uint32_t phase[2] = {0u, 0u};
  bool failed = false;
  int last_stage = -1;

  if (c0 < c1) {
    load_chunk(sA(0), Am, lda, rows, TM, c0 * KC, K);
    load_chunk(sB(0), B, ldb, N, N, c0 * KC, K);
    asm volatile("cp.async.commit_group;\n");
  }
  for (int64_t c = c0; c < c1; ++c) {
    const int st = (int)((c - c0) & 1);
    if (c + 1 < c1) {
      const int nst = st ^ 1;
      if (c > c0) {
        // stage nst held chunk c - 1: its products must be done before reuse
        const bool ok = wait_parity_bounded(&mbar[nst], phase[nst]);
        failed = __syncthreads_or(!ok) != 0;
        if (failed) break;       // last_stage == nst: the wait below retries this phase
        phase[nst] ^= 1u;
      }
      load_chunk(sA(nst), Am, lda, rows, TM, (c + 1) * KC, K);
      load_chunk(sB(nst), B, ldb, N, N, (c + 1) * KC, K);
      asm volatile("cp.async.commit_group;\n");
      asm volatile("cp.async.wait_group 1;\n");
    } else {
      asm volatile("cp.async.wait_group 0;\n");
    }
    asm volatile("fence.proxy.async.shared::cta;\n");
    __syncthreads();
    if (threadIdx.x == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;\n");
#pragma unroll
      for (int ks = 0; ks < KC / 16; ++ks) {
        const uint64_t da = smem_desc(su32(sA(st)) + ks * 256, 128, (KC / 8) * 128);
        const uint64_t db = smem_desc(su32(sB(st)) + ks * 256, 128, (KC / 8) * 128);
        const uint32_t accum = (c > c0 || ks > 0) ? 1u : 0u;
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
            "l"(da), "l"(db), "r"(idesc), "r"(accum));
      }
      asm volatile(
          "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
              su32(&mbar[st])));
    }
    last_stage = st;
  }
  if (!failed && last_stage >= 0) {
    // the last commit covers every product issued before it
    const bool ok = wait_parity_bounded(&mbar[last_stage], phase[last_stage]);
    failed = __syncthreads_or(!ok) != 0;
  }
  if (failed) {
    if (threadIdx.x == 0) atomicCAS(err, 0, 1);
    // give products still in flight a second bounded wait before the TMEM
    // is released, and let the copies land
    if (last_stage >= 0) wait_parity_bounded(&mbar[last_stage], phase[last_stage]);
    asm volatile("cp.async.wait_group 0;\n");
  } else if (last_stage >= 0) {
    asm volatile("tcgen05.fence::after_thread_sync;\n");
    float *out = part + ((size_t)sp * mtiles * TM + (size_t)mt * TM + warp * 32 + lane) * N;
#pragma unroll 1
    for (int cc = 0; cc < N; cc += 16) {
      uint32_t r[16];
      const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)cc;
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
          "%14,%15}, [%16];\n"
          : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
            "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
            "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
          : "r"(taddr));
      asm volatile("tcgen05.wait::ld.sync.aligned;\n");
#pragma unroll
      for (int j = 0; j < 16; j += 4)
        *reinterpret_cast<float4 *>(out + cc + j) =
            make_float4(__uint_as_float(r[j]), __uint_as_float(r[j + 1]),
                        __uint_as_float(r[j + 2]), __uint_as_float(r[j + 3]));
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;\n");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem),
                 "r"(NCOLS));
  }
}

// out[i][j] = sum over splits s (in order) of part[s][i][j], i < Mrows
__global__ void splitk_reduce_kernel(const float *part, int splits, int mtiles, int Mrows, int N,
                                     float *out) {
  const int64_t total = (int64_t)Mrows * N;
  const size_t stride = (size_t)mtiles * TM * N;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total;
       q += (int64_t)gridDim.x * blockDim.x) {
    float acc = 0.f;
    for (int s = 0; s < splits; ++s) acc += part[(size_t)s * stride + q];
    out[q] = acc;
  }
}

template <int N>
cudaError_t launch_splitk(const __nv_bfloat16 *A, int64_t lda, int Mrows, const __nv_bfloat16 *B,
                          int64_t ldb, int64_t K, float *out, float *scratch, size_t scratch_bytes,
                          cudaStream_t st, int *err) {
  constexpr size_t smem = 2 * (size_t)TM * KC * 2 + 2 * (size_t)N * KC * 2 + 32;
  cudaError_t e = cudaFuncSetAttribute(gemm_splitk_tc_kernel<N>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int mtiles = (Mrows + TM - 1) / TM;
  const int64_t nchunks = (K + KC - 1) / KC;
  const size_t per_split = (size_t)mtiles * TM * N * sizeof(float);
  int64_t want = std::max<int64_t>(1, std::min<int64_t>(nchunks, (int64_t)sms / mtiles));
  want = std::min<int64_t>(want, (int64_t)(scratch_bytes / per_split));
  if (want < 1) return cudaErrorInvalidValue;
  const int cps = (int)((nchunks + want - 1) / want);
  const int splits = (int)((nchunks + cps - 1) / cps);
  gemm_splitk_tc_kernel<N><<<splits * mtiles, kTcThreads, smem, st>>>(A, lda, Mrows, B, ldb, K,
                                                                       cps, mtiles, scratch, err);
  const int64_t total = (int64_t)Mrows * N;
  const int rg = (int)std::min<int64_t>((total + 255) / 256, (int64_t)sms * 8);
  splitk_reduce_kernel<<<rg, 256, 0, st>>>(scratch, splits, mtiles, Mrows, N, out);
  note_launches(2);
  return cudaGetLastError();
}

}  // namespace

// Weight-gradient product on tcgen05: out[Mrows x N] (FP32, row-major) =
// A[Mrows x K] . B[N x K]^T, both BF16 K-contiguous (row strides lda, ldb,
// multiples of 8), K any multiple of 8 (the batch), N 64 or 256, Mrows at
// most 256.  The K range is split over CTAs; each writes an FP32 partial to
// `scratch` and a fixed-order sum reduces them (deterministic).  *err
// (device) is set to 1 if a CTA gave up waiting for its products.
cudaError_t gemm_tn_splitk_tc(const __nv_bfloat16 *A, int64_t lda, int Mrows,
                              const __nv_bfloat16 *B, int64_t ldb, int N, int64_t K, float *out,
                              float *scratch, size_t scratch_bytes, cudaStream_t st, int *err) {
  if (K == 0 || Mrows == 0) return cudaSuccess;
  if (lda % 8 || ldb % 8 || K % 8 || !err || Mrows > 256 || ((uintptr_t)scratch % 16))
    return cudaErrorInvalidValue;
  if (N == 256) return launch_splitk<256>(A, lda, Mrows, B, ldb, K, out, scratch, scratch_bytes, st, err);
  if (N == 64) return launch_splitk<64>(A, lda, Mrows, B, ldb, K, out, scratch, scratch_bytes, st, err);
  return cudaErrorNotSupported;
}

}  // namespace pg
