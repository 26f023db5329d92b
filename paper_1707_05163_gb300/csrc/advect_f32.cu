// advect_f32.cu -- FP32 instantiations of the plain advection chunk (FP32
// positions; FP32, FP16 or BF16 field storage).
#include "advect_plain.cuh"
#include "pg_host.h"

namespace pg {

cudaError_t launch_advect_f64(const StepArgs &a, int storage, int block, cudaStream_t st);

template <typename Store, bool SM>
static cudaError_t launch_f32(const StepArgs &a, int block, cudaStream_t st) {
  if (a.p.n == 0) return cudaSuccess;
  const bool d3 = a.g.nz > 1;
  if (a.f.nf == 3)
    return launch_clamped(advect_plain_kernel<float, Store, 3, true, SM>, a, block, st,
                          SM ? corner_smem_bytes(3, true, 1) : 0);
  if (d3)
    return launch_clamped(advect_plain_kernel<float, Store, 2, true, SM>, a, block, st,
                          SM ? corner_smem_bytes(2, true, 1) : 0);
  return launch_clamped(advect_plain_kernel<float, Store, 2, false, SM>, a, block, st,
                        SM ? corner_smem_bytes(2, false, 1) : 0);
}

template <typename Store>
static cudaError_t launch_f32_any(const StepArgs &a, int block, cudaStream_t st, int cache) {
  return cache ? launch_f32<Store, true>(a, block, st) : launch_f32<Store, false>(a, block, st);
}

cudaError_t launch_advect_plain(const StepArgs &a, int real, int storage, int block,
                                cudaStream_t st, int cache) {
  if (real == PG_POS_F64) return launch_advect_f64(a, storage, block, st);
  switch (storage) {
    case PG_F32: return launch_f32_any<float>(a, block, st, cache);
    case PG_F16S: return launch_f32_any<__half>(a, block, st, cache);
    case PG_BF16S: return launch_f32_any<__nv_bfloat16>(a, block, st, cache);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace pg
