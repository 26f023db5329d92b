// moments_noalloc.cu -- FP64 position moments that allocate no memory.
//
// Same reduction as pg_pset_moments, over caller-owned device arrays, for
// callers that must not allocate device memory during a run: processes that
// hand all device memory to their own allocator at start-up (a raw cudaMalloc
// may then fail or fragment that pool), and latency-critical loops where
// cudaMalloc / cudaFree would add host round trips and, for cudaFree, a
// device-wide synchronisation.
//
// The per-block partial sums live in a fixed file-scope device array instead
// of allocated scratch.  Every GPU that loads the library holds that array
// (229,376 bytes) until the process exits.  In host code the array's name is
// only a host-side stand-in, so its device address is looked up once per
// device with cudaGetSymbolAddress and cached.  With lazy module loading the
// first call on a device is also where the array is placed in device memory.
// The cached address belongs to the device's primary context: after
// cudaDeviceReset it is stale, as are all other objects of this library.
#include <mutex>

#include "pg_host.h"

namespace pg {

namespace {

constexpr int kNABlocks = 4096;                 // partial-sum records
constexpr int kNAThreads = 256;
constexpr int64_t kNAPerBlock = 65536;          // particles per block
constexpr int64_t kNAMaxN = (int64_t)kNABlocks * kNAPerBlock;   // 268,435,456

static __device__ __align__(256) double g_na_partial[kNABlocks * 7];

constexpr int kMaxDevices = 64;
std::mutex g_na_mu;
double *g_na_ptr[kMaxDevices] = {nullptr};

// Block b sums particles [b * kNAPerBlock, (b + 1) * kNAPerBlock) in index
// order, thread-strided, then combines its threads in a fixed tree, so the
// result does not depend on timing.  Every block writes its whole record, so
// nothing needs clearing between calls.
__global__ void na_moments_kernel(const double *lon, const double *lat, const double *dep,
                                  const uint8_t *status, int64_t n, double *partial) {
  __shared__ double sh[7][kNAThreads];
  const int64_t beg = (int64_t)blockIdx.x * kNAPerBlock;
  const int64_t end = beg + kNAPerBlock < n ? beg + kNAPerBlock : n;
  double acc[7] = {0, 0, 0, 0, 0, 0, 0};
  for (int64_t p = beg + threadIdx.x; p < end; p += blockDim.x) {
    if (status && status[p] != 0) continue;
    const double a = lon[p], b = lat[p], c = dep ? dep[p] : 0.0;
    acc[0] += 1.0; acc[1] += a; acc[2] += b; acc[3] += c;
    acc[4] += a * a; acc[5] += b * b; acc[6] += c * c;
  }
  for (int q = 0; q < 7; ++q) sh[q][threadIdx.x] = acc[q];
  __syncthreads();
  for (int o = kNAThreads / 2; o > 0; o >>= 1) {
    if (threadIdx.x < (unsigned)o)
      for (int q = 0; q < 7; ++q) sh[q][threadIdx.x] += sh[q][threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0)
    for (int q = 0; q < 7; ++q) partial[(size_t)blockIdx.x * 7 + q] = sh[q][0];
}

__global__ void na_final_kernel(const double *partial, int nblocks, double *out) {
  const int q = threadIdx.x;
  if (q < 7) {
    double s = 0.0;
    for (int b = 0; b < nblocks; ++b) s += partial[(size_t)b * 7 + q];
    out[q] = s;
  }
}

}  // namespace

}  // namespace pg

using namespace pg;

extern "C" pg_status pg_moments_f64_noalloc(const double *lon, const double *lat,
                                            const double *depth, const uint8_t *status,
                                            int64_t n, double *out, void *stream) {
  clear_error();
  if (!lon || !lat || !out) {
    set_error("invalid argument: lon, lat and out must be device pointers");
    return PG_ERR_ARG;
  }
  if (n < 0 || n > kNAMaxN) {
    set_error("invalid argument: n = %lld outside [0, %lld], the limit of the "
              "allocation-free moments", (long long)n, (long long)kNAMaxN);
    return PG_ERR_ARG;
  }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    set_error("cudaGetDevice failed or device %d beyond %d: %s", dev, kMaxDevices,
              cudaGetErrorString(e));
    return PG_ERR_CUDA;
  }
  double *partial = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_na_mu);
    if (!g_na_ptr[dev]) {
      // one-time set-up on this device (the current one)
      void *p = nullptr;
      e = cudaGetSymbolAddress(&p, g_na_partial);
      if (e != cudaSuccess) {
        set_error("cudaGetSymbolAddress of the moments scratch failed: %s",
                  cudaGetErrorString(e));
        return PG_ERR_CUDA;
      }
      g_na_ptr[dev] = (double *)p;
    }
    partial = g_na_ptr[dev];
  }
  cudaStream_t st = (cudaStream_t)stream;
  const int nblocks = (int)((n + kNAPerBlock - 1) / kNAPerBlock);
  if (nblocks > 0)
    na_moments_kernel<<<nblocks, kNAThreads, 0, st>>>(lon, lat, depth, status, n, partial);
  na_final_kernel<<<1, 32, 0, st>>>(partial, nblocks, out);
  note_launches(nblocks > 0 ? 2 : 1);
  e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_error("moments launch failed: %s", cudaGetErrorString(e));
    return PG_ERR_CUDA;
  }
  return PG_OK;
}
