// mlp_fused.cu -- the surrogate network's inference forward in one kernel on
// the 5th-generation tensor cores, activations kept on chip; and, in a
// second instance of the same kernel, a whole network step of the learned
// flow map (features gathered from the field, the network, the displacement
// applied to the particles).
//
// Network: 64 (padded input) -> 256 -> 256 -> 256 -> 256 -> n_out (<= 16;
// the weights are padded to 64 outputs), GELU after the hidden layers (the
// shapes of the flow-map surrogate).  One persistent CTA per SM walks
// 128-row tiles with four kinds of warps working at the same time:
//
//   * input warps fill the tile's input buffer once the previous tile's
//     first layer has read it: two convert FP32 feature rows into BF16 in the
//     operand layout of shared memory (zero-padded to 64 columns); in the
//     network step four gather each particle's 37 features from the field
//     (surrogate_features.cuh), whose loads they wait on;
//   * one lane of a copy warp streams, for every tile, fourteen 32 KB weight
//     pieces -- layer 0; layers 1-3 as four K-quarters each; layer 4 -- into
//     a ring of four slots, each copy completing on the slot's "full"
//     mbarrier;
//   * an MMA warp issues the tcgen05 products into one of two 128 x 256 FP32
//     accumulators in tensor memory (512 columns: layer g uses accumulator
//     g mod 2), each layer as two 128-column halves, and commits "half
//     ready", "slot free" and "input free" mbarriers;
//   * sixteen epilogue warps read an accumulator half back (tcgen05.ld; a
//     warp reaches the 32 lanes -- rows -- of its lane group, four warps per
//     group share the columns), add the bias, apply GELU and write BF16
//     activations into shared memory in the operand layout of the next
//     product; the last layer's 16 columns (plus bias) go to global memory
//     in FP32, or, in the network step, move the particles
//     (surrogate_apply).
//
// The epilogue stores 2 GELU(x) = x (1 + t), one multiply per element fewer
// than GELU(x) = h + h t with h = x / 2, and the packed weights of layers 1-4
// are halved; both scalings are by powers of two and exact in BF16 (for
// normal numbers), so every product and sum is the one of GELU(x) and W, bit
// for bit.
//
// Overlap: the next layer's first two K-quarters need only the first half of
// the activations, so they run while the epilogue works on the second half;
// its first output half is complete (and its epilogue starts) while the
// products of the second half still run; the weight copies run ahead of the
// products by up to four pieces.  The activations live in one 128 x 256
// BF16 buffer: a half is overwritten only after every product that reads it
// has completed (the commits that release an accumulator half cover all
// earlier products).
//
// Every wait is bounded; a warp that gives up raises a CTA-wide flag that
// the others poll, so all leave their loops; then the MMA warp waits
// (bounded) for its products in flight and the copy warp for its copies
// before the tensor memory is released, and *err is set.
//
// Shared-memory operand layout (K-major, no swizzle): 8-row x 16-byte core
// matrices; for a matrix KC 16-byte chunks wide, core (row group g, chunk c)
// sits at byte (g * KC + c) * 128 (descriptor: leading offset 128 bytes,
// stride offset KC * 128 bytes).
#include <cuda_bf16.h>

#include <algorithm>

#include "pg_host.h"
#include "surrogate_features.cuh"

namespace pg {

namespace {

constexpr int TMF = 128;                       // rows per tile
constexpr int kEpiWarps = 16;                  // epilogue warps (a multiple of 4)
constexpr int kCopyWarp = kEpiWarps;
constexpr int kMmaWarp = kEpiWarps + 1;
constexpr int kInWarp0 = kEpiWarps + 2;        // input warps follow the copy and MMA warps
// input warps: two convert feature rows (inference); four gather the
// features of a network step, which wait on field loads
template <bool STEP> struct InWarps { static constexpr int n = STEP ? 4 : 2; };
template <bool STEP> __host__ __device__ constexpr int threads_of() { return 32 * (kEpiWarps + 2 + InWarps<STEP>::n); }
constexpr int kColsPerWarp = 128 / (kEpiWarps / 4);   // of a 128-column half
constexpr long long kFSpin = 4000000;          // mbarrier polls before giving up
constexpr uint32_t kSuspendNs = 500;           // suspend-time hint of a poll
constexpr int kPieces = 14;                    // weight pieces per tile
constexpr uint32_t kPieceBytes = 32768;
constexpr int kSlots = 4;
constexpr uint32_t kTileXBytes = 16384;        // 128 x 64 BF16 input tile
constexpr float kGeluC0 = 0.7978845608028654f;     // sqrt(2 / pi)
constexpr float kGeluC1 = 0.035677408136300125f;   // sqrt(2 / pi) * 0.044715

// shared memory map (bytes)
constexpr uint32_t kOffX = 0;
constexpr uint32_t kOffH = kOffX + kTileXBytes;            // activations, 128 x 256 BF16
constexpr uint32_t kOffW = kOffH + 65536;                  // weight ring
constexpr uint32_t kOffBias = kOffW + kSlots * kPieceBytes;
constexpr uint32_t kBiasFloats = 4 * 256 + 16;
constexpr uint32_t kOffBar = kOffBias + kBiasFloats * 4;
// mbarriers
constexpr int B_WFULL = 0;          // [4] weight slot landed
constexpr int B_WFREE = 4;          // [4] weight slot's products done
constexpr int B_XFULL = 8;          // input tile landed
constexpr int B_XFREE = 9;          // input tile's products done
constexpr int B_ACCFULL = 10;       // [accumulator * 2 + half] products done
constexpr int B_ACCFREE = 14;       // [accumulator * 2 + half] read back
constexpr int B_HFULL = 18;         // [half] activations written
constexpr int B_DRAIN = 20;         // products in flight (failure path)
constexpr int kNumBars = 21;
constexpr uint32_t kOffMisc = kOffBar + kNumBars * 8;      // TMEM address, failure flag
constexpr uint32_t kSmem = kOffMisc + 16;
static_assert(kOffBar % 8 == 0, "mbarrier alignment");
static_assert(kSmem <= 232448, "shared memory per CTA");

__device__ __forceinline__ uint32_t su32f(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ uint64_t desc_f(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((addr & 0x3FFFF) >> 4);
  d |= (uint64_t)((lbo & 0x3FFFF) >> 4) << 16;
  d |= (uint64_t)((sbo & 0x3FFFF) >> 4) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// kind::f16 instruction descriptor: FP32 accumulator, BF16 A and B, both
// K-major, N >> 3 at bit 17, M >> 4 at bit 24.
__host__ __device__ constexpr uint32_t idesc_f(int m, int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) |
         ((uint32_t)(m >> 4) << 24);
}

// Twice GELU in its tanh form, x (1 + tanh(sqrt(2/pi) (x + 0.044715 x^3))),
// as x + x t with the tanh argument x (c0 + c1 x^2); hardware tanh
// approximation.  The layer-by-layer kernels (mlp_tc.cu, mlp.cu) form
// h + h t with h = x / 2 from the same t: exactly half of this value.
__device__ __forceinline__ float gelu2_f(float x) {
  const float p = fmaf(x * x, kGeluC1, kGeluC0);
  float t;
  asm("tanh.approx.f32 %0, %1;" : "=f"(t) : "f"(x * p));
  return fmaf(x, t, x);
}

// Poll phase `parity` of an mbarrier: true once it has completed; false
// after `limit` polls, or (fail != nullptr) once *fail is set.  Each poll may
// suspend the thread for up to kSuspendNs until the phase completes, so a
// waiting warp takes few issue slots from the working ones.
__device__ __forceinline__ bool wait_bar(uint32_t bar, uint32_t parity, const volatile int *fail,
                                         long long limit = kFSpin) {
  for (long long spins = 0; spins < limit; ++spins) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(bar), "r"(parity), "r"(kSuspendNs)
        : "memory");
    if (done) return true;
    if (fail && (spins & 31) == 31 && *fail) return false;
  }
  return false;
}

__device__ __forceinline__ void bar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void bar_expect(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void bulk_copy(uint32_t dst, const void *src, uint32_t bytes,
                                          uint32_t bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
          dst),
      "l"(src), "r"(bytes), "r"(bar)
      : "memory");
}

__device__ __forceinline__ void mma(uint32_t tacc, uint64_t da, uint64_t db, uint32_t idesc,
                                    uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tacc),
      "l"(da), "l"(db), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void commit(uint32_t bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(bar)
      : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&v)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,"
      "%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
        "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
        "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]),
        "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]),
        "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
      : "r"(taddr));
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&v)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,"
      "%15}, [%16];\n"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
        "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
        "=r"(v[14]), "=r"(v[15])
      : "r"(taddr));
}

// Piece p of a tile: its layer, first K element, K length and N.
struct Piece {
  int layer, k0, kl, n;
};
__host__ __device__ __forceinline__ Piece piece_of(int p) {
  Piece q;
  if (p == 0) {
    q.layer = 0; q.k0 = 0; q.kl = 64; q.n = 256;
  } else if (p <= 12) {
    q.layer = (p - 1) / 4 + 1; q.k0 = ((p - 1) % 4) * 64; q.kl = 64; q.n = 256;
  } else {
    q.layer = 4; q.k0 = 0; q.kl = 256; q.n = 64;
  }
  return q;
}

struct FusedArgs {
  const float *x;               // [M x n_in] FP32 features, row-major (inference)
  int n_in;                     // <= 64
  SurrogateStepIO io;           // the particles (network step)
  const uint8_t *wpk;           // packed weight pieces, 32 KB each
  const float *bias[5];         // per layer, N floats
  float *y;                     // [M x n_out] FP32
  int64_t M;
  int n_out;
  int *err;
};

// Row m of the FP32 features into row r of the input buffer: BF16, 64
// columns in the operand layout (core (r / 8, chunk) at ((r / 8) * 8 +
// chunk) * 128 + (r % 8) * 16), zero beyond n_in and for m >= M.  The loads
// of a half row are issued together, so one lane keeps 32 in flight.
__device__ __forceinline__ void load_input_row(const FusedArgs &a, int64_t m, uint8_t *dst, int r) {
  const bool in = m < a.M;
  const float *src = a.x + (in ? m * a.n_in : 0);
  uint8_t *row = dst + (r >> 3) * 1024 + (r & 7) * 16;
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    float f[32];
#pragma unroll
    for (int j = 0; j < 32; ++j) {
      const int col = h * 32 + j;
      f[j] = (in && col < a.n_in) ? __ldg(src + col) : 0.f;
    }
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      uint32_t w[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const __nv_bfloat162 b = __floats2bfloat162_rn(f[c * 8 + 2 * j], f[c * 8 + 2 * j + 1]);
        w[j] = *reinterpret_cast<const uint32_t *>(&b);
      }
      *reinterpret_cast<uint4 *>(row + (h * 4 + c) * 128) = make_uint4(w[0], w[1], w[2], w[3]);
    }
  }
}

// Network step: the features of particle m (zero for a deleted particle or
// m >= M) into row r of the input buffer, as load_input_row lays them out.
__device__ __forceinline__ void feature_row(const FusedArgs &a, int64_t m, uint8_t *dst, int r) {
  float o[kSurFeat];
  bool ok = false;
  if (m < a.M && a.io.status[m] == 0) {
    const int e = surrogate_features(a.io.g, a.io.f, a.io.lon[m], a.io.lat[m], a.io.dep[m],
                                     a.io.time[m], o);
    if (e) atomicCAS(a.io.ferr, 0, e);
    else ok = true;
  }
  uint8_t *row = dst + (r >> 3) * 1024 + (r & 7) * 16;
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    uint32_t w[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int q = c * 8 + 2 * j;
      const float f0 = (ok && q < kSurFeat) ? o[q < kSurFeat ? q : 0] : 0.f;
      const float f1 = (ok && q + 1 < kSurFeat) ? o[q + 1 < kSurFeat ? q + 1 : 0] : 0.f;
      const __nv_bfloat162 h = __floats2bfloat162_rn(f0, f1);
      w[j] = *reinterpret_cast<const uint32_t *>(&h);
    }
    *reinterpret_cast<uint4 *>(row + c * 128) = make_uint4(w[0], w[1], w[2], w[3]);
  }
}

// STEP = false: inference, y = the network on x.  STEP = true: one network
// step of the learned flow map on the particles of a.io.
template <bool STEP>
__global__ void __launch_bounds__(threads_of<STEP>(), 1) mlp_fused_kernel(const __grid_constant__ FusedArgs a) {
  constexpr int kInWarps = InWarps<STEP>::n;
  constexpr int kFThreads = threads_of<STEP>();
  extern __shared__ __align__(1024) uint8_t smem[];
  float *sBias = reinterpret_cast<float *>(smem + kOffBias);
  uint32_t *tslot = reinterpret_cast<uint32_t *>(smem + kOffMisc);
  volatile int *fail = reinterpret_cast<volatile int *>(smem + kOffMisc + 4);
  const uint32_t sbase = su32f(smem);
  const uint32_t sX = sbase + kOffX, sH = sbase + kOffH, sW = sbase + kOffW;
  auto bar = [&](int i) -> uint32_t { return sbase + kOffBar + 8u * (uint32_t)i; };
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t ntiles = (a.M + TMF - 1) / TMF;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                     su32f(tslot)), "r"(512));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
  }
  if (threadIdx.x == 0) {
    for (int i = 0; i < kNumBars; ++i) {
      const uint32_t cnt = (i >= B_ACCFREE && i < B_DRAIN) ? (uint32_t)kEpiWarps
                           : i == B_XFULL ? (uint32_t)kInWarps : 1u;
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(bar(i)), "r"(cnt));
    }
    *fail = 0;
    asm volatile("fence.mbarrier_init.release.cluster;\n");
  }
#pragma unroll
  for (int l = 0; l < 5; ++l)
    for (int i = threadIdx.x; i < (l < 4 ? 256 : 16); i += kFThreads) sBias[l * 256 + i] = a.bias[l][i];
  asm volatile("tcgen05.fence::before_thread_sync;\n");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n");
  const uint32_t tmem = *tslot;
  long long pieces_issued = 0;   // copy warp: for the failure path

  auto give_up = [&]() {
    *fail = 1;
    atomicCAS(a.err, 0, 1);
  };

  if (warp == kCopyWarp) {
    // ------------------------------------------------------ weight copies
    if (lane == 0) {
      long long q = 0;
      bool ok = true;
      for (int64_t tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
        for (int p = 0; p < kPieces; ++p, ++q) {
          const int s = (int)(q & (kSlots - 1));
          if (q >= kSlots && !wait_bar(bar(B_WFREE + s), (uint32_t)(((q / kSlots) - 1) & 1), fail)) {
            ok = false;
            break;
          }
          bar_expect(bar(B_WFULL + s), kPieceBytes);
          const uint8_t *src = a.wpk + (size_t)p * kPieceBytes;
          const uint32_t dst = sW + (uint32_t)s * kPieceBytes;
          bulk_copy(dst, src, 16384, bar(B_WFULL + s));
          bulk_copy(dst + 16384, src + 16384, 16384, bar(B_WFULL + s));
          ++pieces_issued;
        }
      }
      if (!ok) give_up();
    }
  } else if (warp >= kInWarp0) {
    // --------------------------------------------------------- input tiles
    // Tile i's FP32 rows, converted to BF16 in the operand layout, once the
    // previous tile's layer-0 products have read the buffer.
    const int wi = warp - kInWarp0;
    bool ok = true;
    int64_t i = 0;
    for (int64_t tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x, ++i) {
      if (i >= 1) {
        ok = __all_sync(0xffffffffu, wait_bar(bar(B_XFREE), (uint32_t)((i - 1) & 1), fail));
        if (!ok) break;
      }
      for (int r = wi * 32 + lane; r < TMF; r += 32 * kInWarps) {
        if constexpr (STEP) feature_row(a, tile * TMF + r, smem + kOffX, r);
        else load_input_row(a, tile * TMF + r, smem + kOffX, r);
      }
      asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
      __syncwarp();
      if (lane == 0) bar_arrive(bar(B_XFULL));
    }
    if (!ok && lane == 0) give_up();
  } else if (warp == kMmaWarp) {
    // ---------------------------------------------------------- products
    if (lane == 0) {
      long long q = 0;
      uint32_t g = 0;
      int64_t i = 0;
      bool ok = true;
      auto wslot = [&](long long qq) -> uint32_t { return sW + (uint32_t)(qq & (kSlots - 1)) * kPieceBytes; };
      auto wfull = [&](long long qq) -> bool {
        return wait_bar(bar(B_WFULL + (int)(qq & (kSlots - 1))), (uint32_t)((qq / kSlots) & 1), fail);
      };
      auto wfree = [&](long long qq) { commit(bar(B_WFREE + (int)(qq & (kSlots - 1)))); };
      for (int64_t tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x, ++i) {
        for (int L = 0; L < 5 && ok; ++L, ++g) {
          const uint32_t acc = g & 1u, u = g >> 1;
          const uint32_t tacc = tmem + acc * 256u;
          // the accumulator's previous contents (layer g - 2) have been read
          if (u >= 1 && (!wait_bar(bar(B_ACCFREE + 2 * acc), (u - 1) & 1u, fail) ||
                         !wait_bar(bar(B_ACCFREE + 2 * acc + 1), (u - 1) & 1u, fail))) {
            ok = false;
            break;
          }
          if (L == 0) {
            if (!wait_bar(bar(B_XFULL), (uint32_t)(i & 1), fail) || !wfull(q)) { ok = false; break; }
            asm volatile("tcgen05.fence::after_thread_sync;\n");
            for (int nh = 0; nh < 2; ++nh) {
              for (int ks = 0; ks < 4; ++ks)
                mma(tacc + nh * 128, desc_f(sX + ks * 256, 128, 1024),
                    desc_f(wslot(q) + nh * 16384 + ks * 256, 128, 1024), idesc_f(128, 128), ks > 0);
              commit(bar(B_ACCFULL + 2 * acc + nh));
            }
            commit(bar(B_XFREE));
            wfree(q);
            q += 1;
          } else if (L < 4) {
            const uint32_t hp = (uint32_t)((L - 1) & 1);
            // K-quarters 0 and 1 read the first half of the activations
            if (!wait_bar(bar(B_HFULL), hp, fail) || !wfull(q) || !wfull(q + 1)) { ok = false; break; }
            asm volatile("tcgen05.fence::after_thread_sync;\n");
            for (int nh = 0; nh < 2; ++nh)
              for (int kq = 0; kq < 2; ++kq)
                for (int ks = 0; ks < 4; ++ks)
                  mma(tacc + nh * 128, desc_f(sH + kq * 1024 + ks * 256, 128, 4096),
                      desc_f(wslot(q + kq) + nh * 16384 + ks * 256, 128, 1024), idesc_f(128, 128),
                      (kq > 0 || ks > 0) ? 1u : 0u);
            wfree(q);
            wfree(q + 1);
            // K-quarters 2 and 3: the second half
            if (!wait_bar(bar(B_HFULL + 1), hp, fail) || !wfull(q + 2) || !wfull(q + 3)) { ok = false; break; }
            asm volatile("tcgen05.fence::after_thread_sync;\n");
            for (int nh = 0; nh < 2; ++nh) {
              for (int kq = 2; kq < 4; ++kq)
                for (int ks = 0; ks < 4; ++ks)
                  mma(tacc + nh * 128, desc_f(sH + kq * 1024 + ks * 256, 128, 4096),
                      desc_f(wslot(q + kq) + nh * 16384 + ks * 256, 128, 1024), idesc_f(128, 128), 1u);
              commit(bar(B_ACCFULL + 2 * acc + nh));
            }
            wfree(q + 2);
            wfree(q + 3);
            q += 4;
          } else {
            // output layer: N = 16 (the first 16 of the 64 padded rows of W4)
            if (!wait_bar(bar(B_HFULL), 1u, fail) || !wfull(q)) { ok = false; break; }
            asm volatile("tcgen05.fence::after_thread_sync;\n");
            for (int ks = 0; ks < 8; ++ks)
              mma(tacc, desc_f(sH + ks * 256, 128, 4096), desc_f(wslot(q) + ks * 256, 128, 4096),
                  idesc_f(128, 16), ks > 0);
            if (!wait_bar(bar(B_HFULL + 1), 1u, fail)) { ok = false; break; }
            asm volatile("tcgen05.fence::after_thread_sync;\n");
            for (int ks = 8; ks < 16; ++ks)
              mma(tacc, desc_f(sH + ks * 256, 128, 4096), desc_f(wslot(q) + ks * 256, 128, 4096),
                  idesc_f(128, 16), 1u);
            commit(bar(B_ACCFULL + 2 * acc));
            commit(bar(B_ACCFULL + 2 * acc + 1));
            wfree(q);
            q += 1;
          }
        }
      }
      if (!ok) give_up();
      // every product (and every commit before it) has completed before the
      // CTA moves on: bounded, and without the flag so a failing CTA waits too
      commit(bar(B_DRAIN));
      if (!wait_bar(bar(B_DRAIN), 0u, nullptr)) atomicCAS(a.err, 0, 1);
    }
  } else {
    // ---------------------------------------------------------- epilogue
    const int lg = warp & 3, sub = warp >> 2;
    const int r = lg * 32 + lane;
    const uint32_t lane_base = (uint32_t)(lg * 32) << 16;
    uint32_t g = 0;
    bool ok = true;
    for (int64_t tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
      const int64_t m0 = tile * TMF;
      const int rows = (a.M - m0) < TMF ? (int)(a.M - m0) : TMF;
      for (int L = 0; L < 5; ++L, ++g) {
        const uint32_t acc = g & 1u, par = (g >> 1) & 1u;
        if (L < 4) {
          const float *bias = sBias + L * 256;
          for (int h = 0; h < 2; ++h) {
            ok = __all_sync(0xffffffffu, wait_bar(bar(B_ACCFULL + 2 * acc + h), par, fail));
            if (!ok) break;
            asm volatile("tcgen05.fence::after_thread_sync;\n");
            const int c0 = h * 128 + sub * kColsPerWarp;
            uint32_t v[kColsPerWarp];
#pragma unroll
            for (int j = 0; j < kColsPerWarp / 32; ++j)
              tmem_ld32(tmem + lane_base + acc * 256u + (uint32_t)(c0 + 32 * j),
                        *reinterpret_cast<uint32_t(*)[32]>(&v[32 * j]));
            asm volatile("tcgen05.wait::ld.sync.aligned;\n");
            asm volatile("tcgen05.fence::before_thread_sync;\n");
            __syncwarp();
            if (lane == 0) bar_arrive(bar(B_ACCFREE + 2 * acc + h));
            uint8_t *hrow = smem + kOffH + (r >> 3) * 32 * 128 + (r & 7) * 16;
#pragma unroll
            for (int cc = 0; cc < kColsPerWarp; cc += 8) {
              const float4 b0 = *reinterpret_cast<const float4 *>(bias + c0 + cc);
              const float4 b1 = *reinterpret_cast<const float4 *>(bias + c0 + cc + 4);
              const float bb[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
              uint32_t w[4];
#pragma unroll
              for (int j = 0; j < 4; ++j) {
                const float x0 = __uint_as_float(v[cc + 2 * j]) + bb[2 * j];
                const float x1 = __uint_as_float(v[cc + 2 * j + 1]) + bb[2 * j + 1];
                const __nv_bfloat162 hv = __floats2bfloat162_rn(gelu2_f(x0), gelu2_f(x1));
                w[j] = *reinterpret_cast<const uint32_t *>(&hv);
              }
              *reinterpret_cast<uint4 *>(hrow + ((c0 + cc) >> 3) * 128) = make_uint4(w[0], w[1], w[2], w[3]);
            }
            // written by the generic proxy, read by the tensor cores
            asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
            __syncwarp();
            if (lane == 0) bar_arrive(bar(B_HFULL + h));
          }
          if (!ok) break;
        } else {
          ok = __all_sync(0xffffffffu, wait_bar(bar(B_ACCFULL + 2 * acc), par, fail) &&
                                           wait_bar(bar(B_ACCFULL + 2 * acc + 1), par, fail));
          if (!ok) break;
          asm volatile("tcgen05.fence::after_thread_sync;\n");
          uint32_t v[16];
          if (sub == 0) {
            tmem_ld16(tmem + lane_base + acc * 256u, v);
            asm volatile("tcgen05.wait::ld.sync.aligned;\n");
          }
          asm volatile("tcgen05.fence::before_thread_sync;\n");
          __syncwarp();
          if (lane == 0) {
            bar_arrive(bar(B_ACCFREE + 2 * acc));
            bar_arrive(bar(B_ACCFREE + 2 * acc + 1));
          }
          if (sub == 0 && r < rows) {
            const float *bias = sBias + 4 * 256;
            if constexpr (STEP) {
              // the displacement moves the particle (surrogate_apply)
              const int64_t m = m0 + r;
              if (a.io.status[m] == 0) {
                float l = a.io.lon[m], la = a.io.lat[m], d = a.io.dep[m];
                const uint8_t st = surrogate_apply(a.io.g, l, la, d, __uint_as_float(v[0]) + bias[0],
                                                   __uint_as_float(v[1]) + bias[1],
                                                   __uint_as_float(v[2]) + bias[2]);
                if (st) {
                  a.io.status[m] = st;
                } else {
                  a.io.lon[m] = l; a.io.lat[m] = la; a.io.dep[m] = d;
                  a.io.time[m] += a.io.horizon;
                  a.io.step[m] += 1;
                }
              }
            } else {
              float *yr = a.y + (size_t)(m0 + r) * a.n_out;
#pragma unroll
              for (int j = 0; j < 16; ++j)
                if (j < a.n_out) yr[j] = __uint_as_float(v[j]) + bias[j];
            }
          }
        }
      }
    }
    if (!ok) give_up();
  }

  __syncwarp();
  __syncthreads();
  if (*fail && warp == kCopyWarp && lane == 0) {
    // the copies still in flight land before the CTA leaves
    for (long long qq = pieces_issued - 1; qq >= 0 && qq >= pieces_issued - kSlots; --qq)
      wait_bar(bar(B_WFULL + (int)(qq & (kSlots - 1))), (uint32_t)((qq / kSlots) & 1), nullptr);
  }
  __syncwarp();
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;\n");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(512));
  }
}

// A bounded wait on an mbarrier phase that nothing completes (no thread
// arrives on the barrier and no copy or product is in flight): the wait of
// the MLP kernels gives up after `polls` polls, and the block records it in
// *err as those kernels do, then leaves.
__global__ void wait_probe_kernel(long long polls, int *err) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(su32f(&bar)));
    asm volatile("fence.mbarrier_init.release.cluster;\n");
  }
  __syncthreads();
  const bool ok = wait_bar(su32f(&bar), 0u, nullptr, polls);
  if (__syncthreads_or(!ok) && threadIdx.x == 0) atomicCAS(err, 0, 1);
}

// Pack the BF16 weights of the five layers (W_l [dout x din] row-major, as
// mlp.cu keeps them) into the 32 KB pieces of the operand layout; layers 1-4
// halved (their inputs are stored doubled).
__global__ void pack_weights_kernel(const __nv_bfloat16 *w0, const __nv_bfloat16 *w1,
                                    const __nv_bfloat16 *w2, const __nv_bfloat16 *w3,
                                    const __nv_bfloat16 *w4, uint8_t *out) {
  const __nv_bfloat16 *W[5] = {w0, w1, w2, w3, w4};
  for (int p = blockIdx.x; p < kPieces; p += gridDim.x) {
    const Piece q = piece_of(p);
    const int din = q.layer == 0 ? 64 : 256;
    const int kc = q.kl / 8;
    for (int idx = threadIdx.x; idx < q.n * kc; idx += blockDim.x) {
      const int n = idx / kc, c = idx - n * kc;
      uint4 v = *reinterpret_cast<const uint4 *>(W[q.layer] + (size_t)n * din + q.k0 + c * 8);
      if (q.layer > 0) {
        __nv_bfloat162 *h = reinterpret_cast<__nv_bfloat162 *>(&v);
#pragma unroll
        for (int j = 0; j < 4; ++j) h[j] = __hmul2(h[j], __floats2bfloat162_rn(0.5f, 0.5f));
      }
      *reinterpret_cast<uint4 *>(out + (size_t)p * kPieceBytes + ((n >> 3) * kc + c) * 128 +
                                 (n & 7) * 16) = v;
    }
  }
}

}  // namespace

// The bounded-wait probe: one block of 128 threads; *err (device) set to 1
// when the wait gave up.
cudaError_t mlp_wait_probe(long long polls, int *err, cudaStream_t st) {
  wait_probe_kernel<<<1, 128, 0, st>>>(polls, err);
  note_launches(1);
  return cudaGetLastError();
}

// Bytes of the packed weights of the fused forward.
size_t mlp_fused_packed_bytes() { return (size_t)kPieces * kPieceBytes; }

cudaError_t mlp_fused_pack(const __nv_bfloat16 *const w[5], uint8_t *out, cudaStream_t st) {
  pack_weights_kernel<<<kPieces, 256, 0, st>>>(w[0], w[1], w[2], w[3], w[4], out);
  note_launches(1);
  return cudaGetLastError();
}

// y [M x n_out] = the network on x [M x n_in] (FP32 features, n_in <= 64,
// zero-padded to 64 on chip); biases of the five layers (FP32, 256, 256,
// 256, 256, >= n_out entries); *err (device) set to 1 if a CTA gave up
// waiting.
cudaError_t mlp_fused_forward(const float *x, int64_t M, int n_in, const uint8_t *wpk,
                              const float *const bias[5], float *y, int n_out, cudaStream_t st,
                              int *err) {
  if (M == 0) return cudaSuccess;
  if (n_out < 1 || n_out > 16 || n_in < 1 || n_in > 64 || !err || ((uintptr_t)wpk % 16))
    return cudaErrorInvalidValue;
  cudaError_t e = cudaFuncSetAttribute(mlp_fused_kernel<false>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmem);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  FusedArgs a;
  a.x = x; a.n_in = n_in; a.wpk = wpk; a.y = y; a.M = M; a.n_out = n_out; a.err = err;
  for (int l = 0; l < 5; ++l) a.bias[l] = bias[l];
  const int64_t ntiles = (M + TMF - 1) / TMF;
  const int grid = (int)(ntiles < sms ? ntiles : sms);
  mlp_fused_kernel<false><<<grid, threads_of<false>(), kSmem, st>>>(a);
  note_launches(1);
  return cudaGetLastError();
}

// One network step of the learned flow map on io's particles (the network's
// shape: 37 features, 4 x 256, 3 outputs); *err as for mlp_fused_forward,
// feature errors in *io.ferr.
cudaError_t mlp_fused_step_launch(const SurrogateStepIO &io, const uint8_t *wpk,
                                  const float *const bias[5], cudaStream_t st, int *err) {
  if (io.n == 0) return cudaSuccess;
  if (!err || !io.ferr || ((uintptr_t)wpk % 16)) return cudaErrorInvalidValue;
  cudaError_t e = cudaFuncSetAttribute(mlp_fused_kernel<true>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmem);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  FusedArgs a;
  a.x = nullptr; a.n_in = kSurFeat; a.io = io; a.wpk = wpk; a.y = nullptr; a.M = io.n;
  a.n_out = 3; a.err = err;
  for (int l = 0; l < 5; ++l) a.bias[l] = bias[l];
  const int64_t ntiles = (io.n + TMF - 1) / TMF;
  const int grid = (int)(ntiles < sms ? ntiles : sms);
  mlp_fused_kernel<true><<<grid, threads_of<true>(), kSmem, st>>>(a);
  note_launches(1);
  return cudaGetLastError();
}

}  // namespace pg
