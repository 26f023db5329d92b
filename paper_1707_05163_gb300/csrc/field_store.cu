// field_store.cu -- conversion of caller snapshots into the device layout.
//
// Callers give a snapshot planar, [nfields][nz][ny][nx] with lon fastest (the
// layout of one time slice of a FieldSet, Sect. 2.4).  The advection kernels
// read it node-interleaved: node (k, j, i) holds U, V[, W] contiguously
// (three fields padded to four), so one vector load fetches a corner.  For
// FP16/BF16 storage every (field, snapshot) plane gets an FP32 scale
// s = max|v| / 32752 and codes round-to-nearest-even(v / s), with v the FP32
// value of the input.
#include "pg_host.h"

namespace pg {

namespace {

__device__ __forceinline__ float src_value(const void *src, int src_dtype, size_t i) {
  return src_dtype == 0 ? (float)reinterpret_cast<const double *>(src)[i]
                        : reinterpret_cast<const float *>(src)[i];
}

// |v| maxima per field (non-negative floats order like their bit patterns).
__global__ void plane_absmax_kernel(const void *src, int src_dtype, int nf, size_t nodes,
                                    unsigned *amax_bits) {
  const int f = blockIdx.y;
  float m = 0.f;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < nodes;
       i += (size_t)gridDim.x * blockDim.x) {
    const float v = fabsf(src_value(src, src_dtype, (size_t)f * nodes + i));
    m = v > m ? v : m;   // NaN inputs are ignored for the scale
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_down_sync(0xffffffffu, m, o));
  __shared__ float wm[32];
  if ((threadIdx.x & 31) == 0) wm[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x < 32) {
    m = threadIdx.x < (blockDim.x >> 5) ? wm[threadIdx.x] : 0.f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_down_sync(0xffffffffu, m, o));
    if (threadIdx.x == 0) atomicMax(&amax_bits[f], __float_as_uint(m));
  }
}

__global__ void scales_kernel(const unsigned *amax_bits, int nf, float *scales) {
  const int f = threadIdx.x;
  if (f < nf) {
    const float a = __uint_as_float(amax_bits[f]);
    scales[f] = a > 0.f ? a / 32752.0f : 1.0f;
  }
}

template <typename Store>
__device__ __forceinline__ Store to_store(float v, float s);
template <> __device__ __forceinline__ float to_store<float>(float v, float) { return v; }
template <> __device__ __forceinline__ __half to_store<__half>(float v, float s) {
  return __float2half_rn(v / s);
}
template <> __device__ __forceinline__ __nv_bfloat16 to_store<__nv_bfloat16>(float v, float s) {
  return __float2bfloat16_rn(v / s);
}

template <typename Store>
__global__ void repack_kernel(const void *src, int src_dtype, int nf, size_t nodes, Store *dst,
                              const float *scales) {
  const int stride = nf == 2 ? 2 : 4;
  float s[3] = {1.f, 1.f, 1.f};
  if (scales != nullptr)
    for (int f = 0; f < nf; ++f) s[f] = scales[f];
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < nodes;
       i += (size_t)gridDim.x * blockDim.x) {
    for (int f = 0; f < stride; ++f) {
      const float v = f < nf ? src_value(src, src_dtype, (size_t)f * nodes + i) : 0.f;
      dst[i * stride + f] = to_store<Store>(v, f < nf ? s[f] : 1.f);
    }
  }
}

// FP64 storage keeps FP64 input bit for bit.
__global__ void repack_f64_kernel(const void *src, int src_dtype, int nf, size_t nodes,
                                  double *dst) {
  const int stride = nf == 2 ? 2 : 4;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < nodes;
       i += (size_t)gridDim.x * blockDim.x) {
    for (int f = 0; f < stride; ++f) {
      double v = 0.0;
      if (f < nf)
        v = src_dtype == 0 ? reinterpret_cast<const double *>(src)[(size_t)f * nodes + i]
                           : (double)reinterpret_cast<const float *>(src)[(size_t)f * nodes + i];
      dst[i * stride + f] = v;
    }
  }
}

}  // namespace

cudaError_t launch_repack(const void *src, int src_dtype, int nf, size_t nodes, void *dst,
                          int storage, float *scales_out, unsigned *amax_scratch,
                          int sm_count, cudaStream_t st) {
  const int block = 256;
  const size_t want = (nodes + block - 1) / block;
  const int grid = (int)(want < (size_t)sm_count * 8 ? (want ? want : 1) : (size_t)sm_count * 8);
  if (storage == PG_F64) {
    repack_f64_kernel<<<grid, block, 0, st>>>(src, src_dtype, nf, nodes, (double *)dst);
    note_launches(1);
  } else if (storage == PG_F32) {
    repack_kernel<float><<<grid, block, 0, st>>>(src, src_dtype, nf, nodes, (float *)dst, nullptr);
    note_launches(1);
  } else {
    cudaError_t e = cudaMemsetAsync(amax_scratch, 0, sizeof(unsigned) * nf, st);
    if (e != cudaSuccess) return e;
    plane_absmax_kernel<<<dim3(grid, nf), block, 0, st>>>(src, src_dtype, nf, nodes, amax_scratch);
    scales_kernel<<<1, 32, 0, st>>>(amax_scratch, nf, scales_out);
    if (storage == PG_F16S)
      repack_kernel<__half><<<grid, block, 0, st>>>(src, src_dtype, nf, nodes, (__half *)dst,
                                                    scales_out);
    else
      repack_kernel<__nv_bfloat16><<<grid, block, 0, st>>>(src, src_dtype, nf, nodes,
                                                           (__nv_bfloat16 *)dst, scales_out);
    note_launches(3);
  }
  return cudaGetLastError();
}

}  // namespace pg
