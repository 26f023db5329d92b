// probe.cu -- measured read bandwidth of the L2 cache, the denominator of the
// gather kernels' L2 roofline.  A buffer small enough to stay in L2 is read
// with coalesced 16-byte loads that bypass L1 (ld.global.cg), several passes
// per launch, timed with CUDA events after a warm-up; the best of the timed
// launches is reported.
#include "pg_host.h"

namespace pg {

namespace {

__global__ void l2_read_kernel(const float4 *__restrict__ buf, int64_t n, int passes,
                               unsigned *sink) {
  unsigned acc = 0;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int r = 0; r < passes; ++r) {
    // start each pass at a different offset so that no block reads the same
    // lines twice in a row
    const int64_t first = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x +
                           (int64_t)r * blockDim.x * 37) % stride;
    for (int64_t i = first; i < n; i += stride) {
      float4 v;
      asm volatile("ld.global.cg.v4.f32 {%0, %1, %2, %3}, [%4];"
                   : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
                   : "l"(buf + i));
      acc ^= __float_as_uint(v.x) ^ __float_as_uint(v.y) ^ __float_as_uint(v.z) ^
             __float_as_uint(v.w);
    }
  }
  if (acc == 0x9E3779B9u) atomicAdd(sink, 1u);   // keeps the loads; never true for the fill
}

__global__ void fill_probe_kernel(float4 *buf, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    buf[i] = make_float4(1.0f, 2.0f, 3.0f, 4.0f);
}

}  // namespace

}  // namespace pg

using namespace pg;

extern "C" pg_status pg_measure_l2_read(size_t bytes, int reps, double *gbs, void *stream) {
  clear_error();
  if (!gbs || reps < 1 || bytes < ((size_t)1 << 20) || bytes % 16) {
    set_error("invalid argument: need gbs, reps >= 1 and bytes >= 1 MiB, a multiple of 16");
    return PG_ERR_ARG;
  }
  int dev = 0, sms = 0, l2 = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev);
  if (bytes > (size_t)l2 / 2) {
    set_error("invalid argument: %zu bytes do not stay resident in half of the %d-byte L2",
              bytes, l2);
    return PG_ERR_ARG;
  }
  cudaStream_t st = (cudaStream_t)stream;
  float4 *buf = nullptr;
  unsigned *sink = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = dev_alloc((void **)&buf, bytes);
  if (e == cudaSuccess) e = dev_alloc((void **)&sink, 4);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  const int64_t n = (int64_t)(bytes / 16);
  const int passes = 16;
  const int threads = 512, blocks = sms * 4;
  double best = 0.0;
  if (e == cudaSuccess) {
    fill_probe_kernel<<<blocks, threads, 0, st>>>(buf, n);
    l2_read_kernel<<<blocks, threads, 0, st>>>(buf, n, passes, sink);   // warm-up
    note_launches(2);
    e = cudaGetLastError();
  }
  for (int r = 0; r < reps && e == cudaSuccess; ++r) {
    e = cudaEventRecord(e0, st);
    if (e == cudaSuccess) {
      l2_read_kernel<<<blocks, threads, 0, st>>>(buf, n, passes, sink);
      note_launches(1);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(e1, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess && ms > 0.f) best = std::max(best, (double)bytes * passes / (ms * 1e-3) / 1e9);
  }
  cudaStreamSynchronize(st);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  dev_free(buf);
  dev_free(sink);
  if (e != cudaSuccess) {
    set_error("L2 probe failed: %s", cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? PG_ERR_NOMEM : PG_ERR_CUDA;
  }
  *gbs = best;
  return PG_OK;
}
