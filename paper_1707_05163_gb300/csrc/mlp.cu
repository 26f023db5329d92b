// mlp.cu -- the flow-map surrogate's MLP on BF16 tensor cores with FP32
// accumulation: forward (inference and training), backward, Adam.
//
// Network: n_in -> width -> ... (depth hidden layers, GELU) -> n_out.  All
// matrix products are one kernel shape, C[M x N] = A[M x K] . B[N x K]^T with
// both operands K-contiguous BF16 and an FP32 accumulator; the other
// products of back-propagation reach that shape through explicit transposes:
//   forward   Y  = X  W^T      A = X [M x in],      B = W  [out x in]
//   input grad dX = dY W       A = dY [M x out],    B = W^T [in x out]
//   weight grad dW = dY^T X    A = dY^T [out x M],  B = X^T [in x M]
// Widths are padded to multiples of 64 (inputs and outputs zero-padded), so
// every tile is full in N and K; M may be ragged.
//
// GEMM engines: `gemm_nt_mma` uses warp-level mma.sync m16n8k16 (the
// portable tensor-core path); the tcgen05 engine in mlp_tc.cu runs, when
// enabled, every product whose widths are 64 or 256 on Blackwell's
// 5th-generation tensor cores: the forward (bias and GELU in the epilogue),
// the input gradient (GELU' in the epilogue) and the weight gradient (a
// split-K product over the batch).
#include <cuda_bf16.h>

#include <cmath>
#include <cstring>
#include <random>
#include <vector>

#include "pg_host.h"

namespace pg {

// ----------------------------------------------------------------- GEMM ---
namespace {

constexpr int BM = 128, BN = 64, BK = 32;
constexpr int kThreads = 128;   // 4 warps, each 32 rows x 64 columns

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void cp_async16(void *dst, const void *src, bool pred) {
  const int n = pred ? 16 : 0;   // zero-fill out-of-range rows
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(smem_u32(dst)), "l"(src),
               "r"(n));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

__device__ __forceinline__ void ldmatrix_x4(uint32_t &r0, uint32_t &r1, uint32_t &r2, uint32_t &r3,
                                            const void *p) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
               : "r"(smem_u32(p)));
}
__device__ __forceinline__ void ldmatrix_x2(uint32_t &r0, uint32_t &r1, const void *p) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x2.shared.b16 {%0,%1}, [%2];\n"
               : "=r"(r0), "=r"(r1)
               : "r"(smem_u32(p)));
}

__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

}  // namespace

// GELU in its tanh form, 0.5 x (1 + tanh(sqrt(2/pi) (x + 0.044715 x^3))),
// with the hardware tanh approximation (relative error below 2^-10); the
// forward writes it as h + h t with h = x / 2 and the tanh argument
// x (c0 + c1 x^2), the expression of the tcgen05 kernels.
__device__ __forceinline__ float tanh_fast(float x) {
  float y;
  asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float gelu(float x) {
  const float p = fmaf(x * x, 0.035677408136300125f, 0.7978845608028654f);
  const float h = 0.5f * x;
  return fmaf(h, tanh_fast(x * p), h);
}
__device__ __forceinline__ float gelu_grad(float x) {
  const float u = 0.7978845608028654f * (x + 0.044715f * x * x * x);
  const float t = tanh_fast(u);
  return 0.5f * (1.0f + t) +
         0.5f * x * (1.0f - t * t) * 0.7978845608028654f * (1.0f + 0.134145f * x * x);
}

namespace {

// Shared tiles padded by 8 BF16 per row so ldmatrix rows hit distinct banks.
constexpr int SPAD = 8;

struct GemmEpi {
  const float *bias;   // [N] or null
  int act;             // 0 none, 1 GELU
  float *out_f32;      // C in FP32 (or null)
  __nv_bfloat16 *out_bf16;   // C after activation in BF16 (or null)
  __nv_bfloat16 *pre_bf16;   // pre-activation in BF16 (or null)
  int ldc;
  int accumulate;      // out_f32 += C
};

__global__ void __launch_bounds__(kThreads) gemm_nt_mma(const __nv_bfloat16 *__restrict__ A, int lda,
                                                        const __nv_bfloat16 *__restrict__ B, int ldb,
                                                        int M, int N, int K, GemmEpi ep) {
  __shared__ __align__(16) __nv_bfloat16 sA[2][BM][BK + SPAD];
  __shared__ __align__(16) __nv_bfloat16 sB[2][BN][BK + SPAD];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN;
  float acc[2][8][4];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j)
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[i][j][q] = 0.f;

  auto load = [&](int buf, int k0) {
    // A: 128 rows x 32 cols = 512 16-byte chunks, 4 per thread
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int idx = tid + c * kThreads;
      const int r = idx >> 2, col = (idx & 3) * 8;
      const int gr = m0 + r;
      const __nv_bfloat16 *src = A + (size_t)(gr < M ? gr : 0) * lda + k0 + col;
      cp_async16(&sA[buf][r][col], src, gr < M);
    }
    // B: 64 rows x 32 cols = 256 chunks, 2 per thread (N is a multiple of 64)
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      const int idx = tid + c * kThreads;
      const int r = idx >> 2, col = (idx & 3) * 8;
      cp_async16(&sB[buf][r][col], B + (size_t)(n0 + r) * ldb + k0 + col, true);
    }
    cp_async_commit();
  };

  const int nk = K / BK;
  load(0, 0);
  for (int kt = 0; kt < nk; ++kt) {
    const int buf = kt & 1;
    if (kt + 1 < nk) {
      load(buf ^ 1, (kt + 1) * BK);
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; kk += 16) {
      uint32_t af[2][4];
#pragma unroll
      for (int i = 0; i < 2; ++i) {
        const int r = warp * 32 + i * 16 + (lane & 15);
        const int c = kk + (lane >> 4) * 8;
        ldmatrix_x4(af[i][0], af[i][1], af[i][2], af[i][3], &sA[buf][r][c]);
      }
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        uint32_t bf[2];
        const int r = j * 8 + (lane & 7);
        const int c = kk + ((lane >> 3) & 1) * 8;
        ldmatrix_x2(bf[0], bf[1], &sB[buf][r][c]);
#pragma unroll
        for (int i = 0; i < 2; ++i) mma_bf16(acc[i][j], af[i], bf);
      }
    }
    __syncthreads();
  }
  // epilogue: thread holds rows (lane/4, lane/4 + 8) and columns 2*(lane%4) + {0, 1}
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j)
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int row = m0 + warp * 32 + i * 16 + (lane >> 2) + h * 8;
        if (row >= M) continue;
        const int col = n0 + j * 8 + (lane & 3) * 2;
        float v0 = acc[i][j][h * 2 + 0], v1 = acc[i][j][h * 2 + 1];
        if (ep.bias) { v0 += ep.bias[col]; v1 += ep.bias[col + 1]; }
        const size_t o = (size_t)row * ep.ldc + col;
        // column pairs as single 4-byte (BF16) and 8-byte (FP32) stores
        // (col and ldc are even)
        if (ep.pre_bf16)
          *reinterpret_cast<__nv_bfloat162 *>(ep.pre_bf16 + o) = __floats2bfloat162_rn(v0, v1);
        if (ep.act == 1) { v0 = gelu(v0); v1 = gelu(v1); }
        if (ep.out_f32) {
          float2 *d = reinterpret_cast<float2 *>(ep.out_f32 + o);
          if (ep.accumulate) { const float2 c = *d; v0 += c.x; v1 += c.y; }
          *d = make_float2(v0, v1);
        }
        if (ep.out_bf16)
          *reinterpret_cast<__nv_bfloat162 *>(ep.out_bf16 + o) = __floats2bfloat162_rn(v0, v1);
      }
}

// transpose of a BF16 matrix [rows x cols] (row-major) into [cols x rows]
__global__ void transpose_bf16(const __nv_bfloat16 *in, int rows, int cols, int ld_in,
                               __nv_bfloat16 *out, int ld_out) {
  __shared__ __nv_bfloat16 t[32][33];
  const int bx = blockIdx.x * 32, by = blockIdx.y * 32;
  for (int y = threadIdx.y; y < 32; y += blockDim.y) {
    const int r = by + y, c = bx + threadIdx.x;
    t[y][threadIdx.x] = (r < rows && c < cols) ? in[(size_t)r * ld_in + c] : __float2bfloat16(0.f);
  }
  __syncthreads();
  for (int y = threadIdx.y; y < 32; y += blockDim.y) {
    const int c = bx + y, r = by + threadIdx.x;   // out row = c, out col = r
    if (c < cols && r < rows) out[(size_t)c * ld_out + r] = t[threadIdx.x][y];
  }
}

// dPre = dAct * gelu'(pre), both [M x N] (dAct FP32 in, dPre BF16 out), and
// bias gradient partials (column sums) in FP32.
__global__ void gelu_backward(const float *dact, const __nv_bfloat16 *pre, int64_t M, int N,
                              __nv_bfloat16 *dpre, float *dpre_f32) {
  const int64_t total = M * N;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float g = dact[i] * gelu_grad(__bfloat162float(pre[i]));
    dpre[i] = __float2bfloat16_rn(g);
    if (dpre_f32) dpre_f32[i] = g;
  }
}

// column sums of an FP32 [M x N] matrix: one thread per column, fixed order
__global__ void column_sums(const float *x, int64_t M, int N, float *out) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= N) return;
  float s = 0.f;
  for (int64_t r = 0; r < M; ++r) s += x[r * N + c];
  out[c] = s;
}

// BF16 [M x N] -> FP32 copy
__global__ void bf16_to_f32(const __nv_bfloat16 *x, int64_t n, float *y) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    y[i] = __bfloat162float(x[i]);
}

// FP32 [M x n_real] features -> BF16 [M x ld] zero-padded
__global__ void pack_input(const float *x, int64_t M, int n_real, int ld, __nv_bfloat16 *out) {
  const int64_t total = M * ld;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = i / ld;
    const int c = (int)(i - r * ld);
    out[i] = __float2bfloat16_rn(c < n_real ? x[r * n_real + c] : 0.f);
  }
}

// MSE loss 0.5 * mean over rows of sum over the n_out outputs of (y - t)^2
// with output gradient (y - t) / M (FP32, padded columns zero).
__global__ void mse_grad(const float *y, int ldy, const float *t, int n_out, int64_t M,
                         float *dy, float *loss_partial) {
  __shared__ float sh[256];
  float l = 0.f;
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < M;
       r += (int64_t)gridDim.x * blockDim.x) {
    for (int c = 0; c < ldy; ++c) {
      float g = 0.f;
      if (c < n_out) {
        const float d = y[r * ldy + c] - t[r * n_out + c];
        l += 0.5f * d * d;
        g = d / (float)M;
      }
      dy[r * ldy + c] = g;
    }
  }
  sh[threadIdx.x] = l;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < (unsigned)o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) loss_partial[blockIdx.x] = sh[0];
}

__global__ void f32_to_bf16(const float *x, int64_t n, __nv_bfloat16 *y) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    y[i] = __float2bfloat16_rn(x[i]);
}

// Adam on FP32 master parameters; refreshes the BF16 weights [out x in] and
// their transposes [in x out] for the real (unpadded) block.
struct AdamArgs {
  float *w, *m, *v;
  const float *g;
  int64_t n;
  float lr, b1, b2, eps, c1, c2;   // c1 = 1 / (1 - b1^t), c2 = 1 / (1 - b2^t)
};
__global__ void adam_kernel(AdamArgs a) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float g = a.g[i];
    const float m = a.b1 * a.m[i] + (1.f - a.b1) * g;
    const float v = a.b2 * a.v[i] + (1.f - a.b2) * g * g;
    a.m[i] = m;
    a.v[i] = v;
    a.w[i] -= a.lr * (m * a.c1) / (sqrtf(v * a.c2) + a.eps);
  }
}

int grid1(int64_t n) {
  int64_t g = (n + 255) / 256;
  if (g > 4096) g = 4096;
  return (int)(g < 1 ? 1 : g);
}

}  // namespace

cudaError_t gemm_nt(const __nv_bfloat16 *A, int lda, const __nv_bfloat16 *B, int ldb, int64_t M,
                    int N, int K, const float *bias, int act, float *out_f32,
                    __nv_bfloat16 *out_bf16, __nv_bfloat16 *pre_bf16, int ldc, int accumulate,
                    cudaStream_t st) {
  if (M == 0) return cudaSuccess;
  if (N % BN || K % BK || ldc % 2) return cudaErrorInvalidValue;
  if (((uintptr_t)out_f32 % 8) || ((uintptr_t)out_bf16 % 4) || ((uintptr_t)pre_bf16 % 4))
    return cudaErrorInvalidValue;
  GemmEpi ep{bias, act, out_f32, out_bf16, pre_bf16, ldc, accumulate};
  dim3 grid((unsigned)((M + BM - 1) / BM), (unsigned)(N / BN));
  gemm_nt_mma<<<grid, kThreads, 0, st>>>(A, lda, B, ldb, (int)M, N, K, ep);
  note_launches(1);
  return cudaGetLastError();
}

}  // namespace pg

// ------------------------------------------------------------ the network --

using namespace pg;

struct pg_mlp {
  int n_in, width, depth, n_out;
  int pin, pout;                      // padded input / output widths (multiples of 64)
  int nl;                             // layers = depth + 1
  std::vector<int> din, dout;         // padded dims per layer
  // FP32 master parameters, Adam moments, gradients: one buffer each,
  // layer l's W [dout x din] then b [dout]
  std::vector<size_t> woff, boff;
  size_t nparam = 0;
  float *w = nullptr, *m = nullptr, *v = nullptr, *g = nullptr;
  __nv_bfloat16 *wb = nullptr;        // BF16 W [dout x din] per layer (same offsets)
  __nv_bfloat16 *wbt = nullptr;       // BF16 W^T [din x dout]
  int64_t step = 0;
  // workspace for a batch of up to cap rows
  int64_t cap = 0;
  __nv_bfloat16 *x0 = nullptr;        // packed input [cap x pin]
  std::vector<__nv_bfloat16 *> act;   // post-activation per hidden layer [cap x width]
  std::vector<__nv_bfloat16 *> pre;   // pre-activation per hidden layer
  float *y = nullptr;                 // output [cap x pout] FP32
  float *dy = nullptr;                // FP32 gradient of the current layer output [cap x width]
  __nv_bfloat16 *dyb = nullptr, *dyt = nullptr, *xt = nullptr;   // BF16 grads, transposes
  __nv_bfloat16 *dyb2 = nullptr;      // second BF16 gradient buffer (tcgen05 input gradient)
  float *gscratch = nullptr;          // split-K partials of the weight gradient
  size_t gscratch_bytes = 0;
  float *loss_partial = nullptr;
  int use_tc = 0;                     // tcgen05 products when available
  int fused = 1;                      // tcgen05 inference in one fused kernel when the shape allows
  uint8_t *wpk = nullptr;             // weights packed for the fused forward
  bool wpk_valid = false;
  int *d_err = nullptr;               // device word: tcgen05 wait gave up
};

namespace pg {
cudaError_t gemm_nt_tc(const __nv_bfloat16 *A, int lda, const __nv_bfloat16 *B, int ldb,
                       int64_t M, int N, int K, const float *bias, int act, float *out_f32,
                       __nv_bfloat16 *out_bf16, __nv_bfloat16 *pre_bf16, int ldc, cudaStream_t st,
                       int *err, const __nv_bfloat16 *gin = nullptr);
size_t mlp_fused_packed_bytes();
cudaError_t mlp_fused_pack(const __nv_bfloat16 *const w[5], uint8_t *out, cudaStream_t st);
cudaError_t mlp_fused_forward(const float *x, int64_t M, int n_in, const uint8_t *wpk,
                              const float *const bias[5], float *y, int n_out, cudaStream_t st,
                              int *err);
cudaError_t mlp_fused_step_launch(const SurrogateStepIO &io, const uint8_t *wpk,
                                  const float *const bias[5], cudaStream_t st, int *err);
cudaError_t mlp_wait_probe(long long polls, int *err, cudaStream_t st);
cudaError_t gemm_tn_splitk_tc(const __nv_bfloat16 *A, int64_t lda, int Mrows,
                              const __nv_bfloat16 *B, int64_t ldb, int N, int64_t K, float *out,
                              float *scratch, size_t scratch_bytes, cudaStream_t st, int *err);
}

namespace {

void free_ws(pg_mlp *n) {
  dev_free(n->x0);
  for (auto p : n->act) dev_free(p);
  for (auto p : n->pre) dev_free(p);
  n->act.clear();
  n->pre.clear();
  dev_free(n->y); dev_free(n->dy); dev_free(n->dyb); dev_free(n->dyt); dev_free(n->xt);
  dev_free(n->dyb2); dev_free(n->gscratch);
  n->dyb2 = nullptr; n->gscratch = nullptr; n->gscratch_bytes = 0;
  dev_free(n->loss_partial);
  n->x0 = nullptr; n->y = nullptr; n->dy = nullptr; n->dyb = nullptr; n->dyt = nullptr;
  n->xt = nullptr; n->loss_partial = nullptr;
  n->cap = 0;
}

cudaError_t ensure_ws(pg_mlp *n, int64_t rows) {
  if (rows <= n->cap) return cudaSuccess;
  free_ws(n);
  const int64_t cap = rows;
  cudaError_t e = cudaSuccess;
  auto al = [&](void **p, size_t b) {
    if (e == cudaSuccess) e = dev_alloc(p, b);
  };
  al((void **)&n->x0, cap * n->pin * 2);
  for (int l = 0; l < n->depth; ++l) {
    __nv_bfloat16 *a = nullptr, *p = nullptr;
    al((void **)&a, cap * n->width * 2);
    al((void **)&p, cap * n->width * 2);
    n->act.push_back(a);
    n->pre.push_back(p);
  }
  const int wmax = std::max(n->width, n->pout);
  al((void **)&n->y, cap * n->pout * 4);
  al((void **)&n->dy, cap * wmax * 4);
  al((void **)&n->dyb, cap * wmax * 2);
  al((void **)&n->dyb2, cap * wmax * 2);
  // split-K partials: up to 64 splits of a 256 x 256 product
  n->gscratch_bytes = (size_t)64 * 256 * 256 * sizeof(float);
  al((void **)&n->gscratch, n->gscratch_bytes);
  al((void **)&n->dyt, cap * wmax * 2);
  al((void **)&n->xt, cap * std::max(n->width, n->pin) * 2);
  al((void **)&n->loss_partial, 1024 * 4);
  if (e != cudaSuccess) {
    free_ws(n);
    return e;
  }
  n->cap = cap;
  return cudaSuccess;
}

// BF16 copies of the weights and of their transposes from the FP32 masters
cudaError_t refresh_bf16(pg_mlp *n, cudaStream_t st) {
  n->wpk_valid = false;
  f32_to_bf16<<<grid1((int64_t)n->nparam), 256, 0, st>>>(n->w, (int64_t)n->nparam, n->wb);
  note_launches(1);
  for (int l = 0; l < n->nl; ++l) {
    dim3 g((n->din[l] + 31) / 32, (n->dout[l] + 31) / 32);
    transpose_bf16<<<g, dim3(32, 8), 0, st>>>(n->wb + n->woff[l], n->dout[l], n->din[l], n->din[l],
                                              n->wbt + n->woff[l], n->dout[l]);
    note_launches(1);
  }
  return cudaGetLastError();
}

// forward through all layers for `rows` packed inputs in n->x0; keeps the
// pre/post activations for the backward pass
cudaError_t forward(pg_mlp *n, int64_t rows, cudaStream_t st, bool keep) {
  const __nv_bfloat16 *x = n->x0;
  int ldx = n->pin;
  for (int l = 0; l < n->nl; ++l) {
    const bool last = l == n->nl - 1;
    const __nv_bfloat16 *W = n->wb + n->woff[l];
    const float *b = n->w + n->boff[l];
    cudaError_t e;
    const bool tc_shape = (n->dout[l] == 64 || n->dout[l] == 256) &&
                          (n->din[l] == 64 || n->din[l] == 256);
    if (n->use_tc && tc_shape) {
      e = gemm_nt_tc(x, ldx, W, n->din[l], rows, n->dout[l], n->din[l], b, last ? 0 : 1,
                     last ? n->y : nullptr, last ? nullptr : n->act[l],
                     (!last && keep) ? n->pre[l] : nullptr, n->dout[l], st, n->d_err);
    } else {
      e = gemm_nt(x, ldx, W, n->din[l], rows, n->dout[l], n->din[l], b, last ? 0 : 1,
                  last ? n->y : nullptr, last ? nullptr : n->act[l],
                  (!last && keep) ? n->pre[l] : nullptr, n->dout[l], 0, st);
    }
    if (e != cudaSuccess) return e;
    if (!last) {
      x = n->act[l];
      ldx = n->width;
    }
  }
  return cudaSuccess;
}

// backward from n->dy (gradient of the FP32 output, [rows x pout]) into n->g
cudaError_t backward(pg_mlp *n, int64_t rows, cudaStream_t st) {
  cudaError_t e;
  // gradient w.r.t. the current layer's pre-activation (BF16 copy in dyb)
  int wcur = n->pout;
  f32_to_bf16<<<grid1(rows * wcur), 256, 0, st>>>(n->dy, rows * wcur, n->dyb);
  note_launches(1);
  for (int l = n->nl - 1; l >= 0; --l) {
    const __nv_bfloat16 *X = l == 0 ? n->x0 : n->act[l - 1];
    const int din = n->din[l], dout = n->dout[l];
    // bias gradient: column sums of dPre (FP32, in dy)
    column_sums<<<(dout + 127) / 128, 128, 0, st>>>(n->dy, rows, dout, n->g + n->boff[l]);
    // dW [dout x din] = dPre^T X: transposes to K-contiguous [dout x rows], [din x rows]
    dim3 g1((dout + 31) / 32, (unsigned)((rows + 31) / 32));
    transpose_bf16<<<g1, dim3(32, 8), 0, st>>>(n->dyb, (int)rows, dout, dout, n->dyt, (int)rows);
    dim3 g2((din + 31) / 32, (unsigned)((rows + 31) / 32));
    transpose_bf16<<<g2, dim3(32, 8), 0, st>>>(X, (int)rows, din, din, n->xt, (int)rows);
    note_launches(3);
    const bool tc = n->use_tc && (din == 64 || din == 256) && (dout == 64 || dout == 256);
    // rows must be a multiple of 32 for the K loop; the batch is padded
    if (tc) e = gemm_tn_splitk_tc(n->dyt, rows, dout, n->xt, rows, din, rows, n->g + n->woff[l],
                                  n->gscratch, n->gscratch_bytes, st, n->d_err);
    else e = gemm_nt(n->dyt, (int)rows, n->xt, (int)rows, dout, din, (int)rows, nullptr, 0,
                     n->g + n->woff[l], nullptr, nullptr, din, 0, st);
    if (e != cudaSuccess) return e;
    if (l == 0) break;
    if (tc) {
      // dPre of layer l-1 = (dPre W) * GELU'(pre) in one product (B = W^T
      // [din x dout]); FP32 into dy, BF16 into the other buffer (the one
      // read as A must not be overwritten by other tiles)
      if ((e = gemm_nt_tc(n->dyb, dout, n->wbt + n->woff[l], dout, rows, din, dout, nullptr, 2,
                          n->dy, n->dyb2, nullptr, din, st, n->d_err, n->pre[l - 1])) !=
          cudaSuccess)
        return e;
      std::swap(n->dyb, n->dyb2);
    } else {
      // dX [rows x din] = dPre W  (B = W^T [din x dout])
      if ((e = gemm_nt(n->dyb, dout, n->wbt + n->woff[l], dout, rows, din, dout, nullptr, 0, n->dy,
                       nullptr, nullptr, din, 0, st)) != cudaSuccess)
        return e;
      // through the GELU of layer l-1
      gelu_backward<<<grid1(rows * din), 256, 0, st>>>(n->dy, n->pre[l - 1], rows, din, n->dyb,
                                                       n->dy);
      note_launches(1);
    }
    wcur = din;
  }
  return cudaGetLastError();
}

int round64(int x) { return (x + 63) / 64 * 64; }

}  // namespace

#define CUM(call)                                                                     \
  do {                                                                                \
    cudaError_t e_ = (call);                                                          \
    if (e_ != cudaSuccess) {                                                          \
      set_error("%s failed: %s", #call, cudaGetErrorString(e_));                      \
      return e_ == cudaErrorMemoryAllocation ? PG_ERR_NOMEM : PG_ERR_CUDA;            \
    }                                                                                 \
  } while (0)

namespace pg {

// The fused kernel's shape: inputs padded to 64, four hidden layers of 256,
// outputs padded to 64 with at most 16 real ones.
static bool fused_shape(const pg_mlp *n) {
  return n->use_tc && n->fused && n->pin == 64 && n->width == 256 && n->depth == 4 &&
         n->pout == 64 && n->n_out <= 16;
}

static cudaError_t ensure_packed(pg_mlp *n, cudaStream_t st) {
  if (n->wpk_valid) return cudaSuccess;
  const __nv_bfloat16 *w[5];
  for (int l = 0; l < 5; ++l) w[l] = n->wb + n->woff[l];
  cudaError_t e = mlp_fused_pack(w, n->wpk, st);
  if (e == cudaSuccess) n->wpk_valid = true;
  return e;
}

bool mlp_fused_step_ok(const pg_mlp *n) { return n && fused_shape(n) && n->n_in == 37 && n->n_out == 3; }

pg_status mlp_fused_step(pg_mlp *n, const SurrogateStepIO &io, cudaStream_t st) {
  if (!mlp_fused_step_ok(n)) { set_error("network cannot run the fused step"); return PG_ERR_ARG; }
  CUM(ensure_packed(n, st));
  const float *bias[5];
  for (int l = 0; l < 5; ++l) bias[l] = n->w + n->boff[l];
  CUM(cudaMemsetAsync(io.ferr, 0, 4, st));
  CUM(mlp_fused_step_launch(io, n->wpk, bias, st, n->d_err));
  int err[2] = {0, 0};
  CUM(cudaMemcpyAsync(&err[0], n->d_err, 4, cudaMemcpyDeviceToHost, st));
  CUM(cudaMemcpyAsync(&err[1], io.ferr, 4, cudaMemcpyDeviceToHost, st));
  CUM(cudaStreamSynchronize(st));
  if (err[0]) { set_error("tcgen05 product gave up waiting for its accumulator"); return PG_ERR_TIMEOUT; }
  if (err[1]) { set_error("feature gather recorded internal error %d", err[1]); return PG_ERR_DEVICE; }
  return PG_OK;
}

}  // namespace pg

extern "C" {

pg_status pg_mlp_create(int n_in, int width, int depth, int n_out, uint64_t seed, pg_mlp **out) {
  clear_error();
  if (!out || n_in < 1 || n_in > 1024 || width < 64 || width % 64 || width > 1024 || depth < 1 ||
      depth > 16 || n_out < 1 || n_out > 64) {
    set_error("invalid argument: need 1 <= n_in <= 1024, width a multiple of 64 in [64, 1024], "
              "1 <= depth <= 16, 1 <= n_out <= 64");
    return PG_ERR_ARG;
  }
  auto *n = new pg_mlp();
  n->n_in = n_in; n->width = width; n->depth = depth; n->n_out = n_out;
  n->pin = round64(n_in);
  n->pout = round64(n_out);
  n->nl = depth + 1;
  for (int l = 0; l < n->nl; ++l) {
    n->din.push_back(l == 0 ? n->pin : width);
    n->dout.push_back(l == n->nl - 1 ? n->pout : width);
  }
  size_t off = 0;
  for (int l = 0; l < n->nl; ++l) {
    n->woff.push_back(off);
    off += (size_t)n->din[l] * n->dout[l];
    n->boff.push_back(off);
    off += n->dout[l];
  }
  n->nparam = off;
  // He-style uniform initialisation of the real block, zeros in the padding
  std::vector<float> h(off, 0.f);
  std::mt19937_64 rng(seed);
  for (int l = 0; l < n->nl; ++l) {
    const int rin = l == 0 ? n_in : width, rout = l == n->nl - 1 ? n_out : width;
    const float lim = std::sqrt(6.0f / (float)rin) * (l == n->nl - 1 ? 0.1f : 1.0f);
    std::uniform_real_distribution<float> U(-lim, lim);
    for (int o = 0; o < rout; ++o)
      for (int i = 0; i < rin; ++i) h[n->woff[l] + (size_t)o * n->din[l] + i] = U(rng);
  }
  cudaError_t e = dev_alloc((void **)&n->w, off * 4);
  if (e == cudaSuccess) e = dev_alloc((void **)&n->m, off * 4);
  if (e == cudaSuccess) e = dev_alloc((void **)&n->v, off * 4);
  if (e == cudaSuccess) e = dev_alloc((void **)&n->g, off * 4);
  if (e == cudaSuccess) e = dev_alloc((void **)&n->wb, off * 2);
  if (e == cudaSuccess) e = dev_alloc((void **)&n->wbt, off * 2);
  if (e == cudaSuccess) e = dev_alloc((void **)&n->d_err, 4);
  if (e == cudaSuccess) e = cudaMemset(n->d_err, 0, 4);
  if (e == cudaSuccess) e = dev_alloc((void **)&n->wpk, mlp_fused_packed_bytes());
  if (e == cudaSuccess) e = cudaMemcpy(n->w, h.data(), off * 4, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(n->m, 0, off * 4);
  if (e == cudaSuccess) e = cudaMemset(n->v, 0, off * 4);
  if (e == cudaSuccess) e = cudaMemset(n->g, 0, off * 4);
  if (e == cudaSuccess) e = refresh_bf16(n, 0);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    dev_free(n->w); dev_free(n->m); dev_free(n->v); dev_free(n->g); dev_free(n->wb);
    dev_free(n->wbt);
    dev_free(n->d_err);
    delete n;
    cudaGetLastError();
    set_error("MLP allocation failed: %s", cudaGetErrorString(e));
    return PG_ERR_NOMEM;
  }
  *out = n;
  return PG_OK;
}

pg_status pg_mlp_destroy(pg_mlp *n) {
  if (!n) return PG_OK;
  cudaDeviceSynchronize();
  free_ws(n);
  dev_free(n->w); dev_free(n->m); dev_free(n->v); dev_free(n->g); dev_free(n->wb);
  dev_free(n->wbt);
  dev_free(n->d_err);
  dev_free(n->wpk);
  delete n;
  return PG_OK;
}

pg_status pg_mlp_num_params(const pg_mlp *n, int64_t *padded, int64_t *real) {
  clear_error();
  if (!n) { set_error("invalid argument: null network"); return PG_ERR_ARG; }
  if (padded) *padded = (int64_t)n->nparam;
  if (real) {
    int64_t r = 0;
    for (int l = 0; l < n->nl; ++l) {
      const int rin = l == 0 ? n->n_in : n->width, rout = l == n->nl - 1 ? n->n_out : n->width;
      r += (int64_t)rin * rout + rout;
    }
    *real = r;
  }
  return PG_OK;
}

// Parameters in the padded layout (layer l: W [dout x din] row-major, then
// b [dout]) as FP32, host memory of pg_mlp_num_params().padded floats.
pg_status pg_mlp_get_params(const pg_mlp *n, float *host) {
  clear_error();
  if (!n || !host) { set_error("invalid argument"); return PG_ERR_ARG; }
  CUM(cudaMemcpy(host, n->w, n->nparam * 4, cudaMemcpyDeviceToHost));
  return PG_OK;
}

pg_status pg_mlp_set_params(pg_mlp *n, const float *host) {
  clear_error();
  if (!n || !host) { set_error("invalid argument"); return PG_ERR_ARG; }
  CUM(cudaMemcpy(n->w, host, n->nparam * 4, cudaMemcpyHostToDevice));
  CUM(refresh_bf16(n, 0));
  CUM(cudaDeviceSynchronize());
  return PG_OK;
}

pg_status pg_mlp_set_engine(pg_mlp *n, int tcgen05) {
  clear_error();
  if (!n || tcgen05 < 0 || tcgen05 > 2) { set_error("invalid argument"); return PG_ERR_ARG; }
  n->use_tc = tcgen05 ? 1 : 0;
  n->fused = tcgen05 == 1 ? 1 : 0;
  return PG_OK;
}

// Forward: x [M x n_in] FP32 device -> y [M x n_out] FP32 device.
pg_status pg_mlp_forward(pg_mlp *n, const float *x, int64_t M, float *y, void *stream) {
  clear_error();
  if (!n || (M > 0 && (!x || !y)) || M < 0) { set_error("invalid argument"); return PG_ERR_ARG; }
  cudaStream_t st = (cudaStream_t)stream;
  const int64_t chunk = 1 << 20;
  // the surrogate's shape runs as one fused tcgen05 kernel (activations on chip)
  const bool fused = fused_shape(n);
  if (fused) CUM(ensure_packed(n, st));
  if (fused) {
    // one launch over all rows: the kernel reads the FP32 features itself
    // and needs no workspace
    const float *bias[5];
    for (int l = 0; l < 5; ++l) bias[l] = n->w + n->boff[l];
    CUM(mlp_fused_forward(x, M, n->n_in, n->wpk, bias, y, n->n_out, st, n->d_err));
  }
  for (int64_t r0 = 0; r0 < M && !fused; r0 += chunk) {
    const int64_t rows = std::min(chunk, M - r0);
    CUM(ensure_ws(n, std::min<int64_t>(M, chunk)));
    pack_input<<<grid1(rows * n->pin), 256, 0, st>>>(x + r0 * n->n_in, rows, n->n_in, n->pin, n->x0);
    note_launches(1);
    CUM(forward(n, rows, st, false));
    CUM(cudaMemcpy2DAsync(y + r0 * n->n_out, n->n_out * 4, n->y, n->pout * 4, n->n_out * 4, rows,
                          cudaMemcpyDeviceToDevice, st));
  }
  CUM(cudaGetLastError());
  if (n->use_tc) {
    int err = 0;
    CUM(cudaMemcpyAsync(&err, n->d_err, 4, cudaMemcpyDeviceToHost, st));
    CUM(cudaStreamSynchronize(st));
    if (err) {
      set_error("tcgen05 product gave up waiting for its accumulator");
      return PG_ERR_TIMEOUT;
    }
  }
  return PG_OK;
}

// Gradient of L = 0.5 * mean_rows sum_out (y - t)^2 with respect to every
// parameter (padded layout), into host `grad` (may be NULL) and the internal
// gradient buffer; loss to *loss.  M must be a multiple of 32.
static pg_status mlp_grad_impl(pg_mlp *n, const float *x, const float *t, int64_t M, float *loss,
                               cudaStream_t st) {
  if (M % 32) { set_error("invalid argument: batch size must be a multiple of 32"); return PG_ERR_ARG; }
  CUM(ensure_ws(n, M));
  pack_input<<<grid1(M * n->pin), 256, 0, st>>>(x, M, n->n_in, n->pin, n->x0);
  note_launches(1);
  CUM(forward(n, M, st, true));
  const int nb = (int)std::min<int64_t>(1024, (M + 255) / 256);
  mse_grad<<<nb, 256, 0, st>>>(n->y, n->pout, t, n->n_out, M, n->dy, n->loss_partial);
  note_launches(1);
  CUM(cudaMemsetAsync(n->g, 0, n->nparam * 4, st));
  CUM(backward(n, M, st));
  if (n->use_tc) {
    int err = 0;
    CUM(cudaMemcpyAsync(&err, n->d_err, 4, cudaMemcpyDeviceToHost, st));
    CUM(cudaStreamSynchronize(st));
    if (err) {
      set_error("a tcgen05 product gave up waiting for its accumulator");
      return PG_ERR_TIMEOUT;
    }
  }
  if (loss) {
    std::vector<float> lp(nb);
    CUM(cudaMemcpyAsync(lp.data(), n->loss_partial, nb * 4, cudaMemcpyDeviceToHost, st));
    CUM(cudaStreamSynchronize(st));
    double s = 0;
    for (float v : lp) s += v;
    *loss = (float)(s / (double)M);
  }
  return PG_OK;
}

pg_status pg_mlp_grad(pg_mlp *n, const float *x, const float *t, int64_t M, float *loss,
                      float *grad_host, void *stream) {
  clear_error();
  if (!n || !x || !t || M <= 0) { set_error("invalid argument"); return PG_ERR_ARG; }
  cudaStream_t st = (cudaStream_t)stream;
  pg_status r = mlp_grad_impl(n, x, t, M, loss, st);
  if (r) return r;
  if (grad_host) {
    CUM(cudaMemcpyAsync(grad_host, n->g, n->nparam * 4, cudaMemcpyDeviceToHost, st));
    CUM(cudaStreamSynchronize(st));
  }
  return PG_OK;
}

// One Adam step on a batch (x [M x n_in], targets t [M x n_out], device).
pg_status pg_mlp_train_step(pg_mlp *n, const float *x, const float *t, int64_t M, float lr,
                            float *loss, void *stream) {
  clear_error();
  if (!n || !x || !t || M <= 0) { set_error("invalid argument"); return PG_ERR_ARG; }
  cudaStream_t st = (cudaStream_t)stream;
  pg_status r = mlp_grad_impl(n, x, t, M, loss, st);
  if (r) return r;
  n->step += 1;
  const float b1 = 0.9f, b2 = 0.999f;
  AdamArgs a{n->w, n->m, n->v, n->g, (int64_t)n->nparam, lr, b1, b2, 1e-8f,
             (float)(1.0 / (1.0 - std::pow((double)b1, (double)n->step))),
             (float)(1.0 / (1.0 - std::pow((double)b2, (double)n->step)))};
  adam_kernel<<<grid1((int64_t)n->nparam), 256, 0, st>>>(a);
  note_launches(1);
  CUM(refresh_bf16(n, st));
  return PG_OK;
}

// The bounded mbarrier wait of the tcgen05 kernels, run on a phase nothing
// completes (test hook).
pg_status pg_debug_bounded_wait(int64_t polls, void *stream) {
  clear_error();
  if (polls < 1 || polls > 10000000) { set_error("invalid argument: polls in [1, 1e7]"); return PG_ERR_ARG; }
  cudaStream_t st = (cudaStream_t)stream;
  int *d = nullptr;
  CUM(dev_alloc((void **)&d, 4));
  int h = 0;
  cudaError_t e = cudaMemsetAsync(d, 0, 4, st);
  if (e == cudaSuccess) e = mlp_wait_probe((long long)polls, d, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h, d, 4, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  dev_free(d);
  CUM(e);
  if (h) {
    set_error("bounded wait gave up after %lld polls", (long long)polls);
    return PG_ERR_TIMEOUT;
  }
  return PG_OK;
}

}  // extern "C"
