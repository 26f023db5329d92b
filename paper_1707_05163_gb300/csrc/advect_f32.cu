// advect_f32.cu -- FP32 instantiations of the plain advection chunk (FP32
// positions; FP32, FP16 or BF16 field storage).
#include "advect_plain.cuh"
#include "pg_host.h"

namespace pg {

cudaError_t launch_advect_f64(const StepArgs &a, int storage, int block, cudaStream_t st);

template <typename Store, int GEO>
static cudaError_t launch_geo(const StepArgs &a, int block, cudaStream_t st) {
  if (a.f.nf == 3) return launch_clamped<advect_plain_kernel<float, Store, 3, true, GEO>>(a, block, st);
  if (a.g.nz > 1) return launch_clamped<advect_plain_kernel<float, Store, 2, true, GEO>>(a, block, st);
  return launch_clamped<advect_plain_kernel<float, Store, 2, false, GEO>>(a, block, st);
}

template <typename Store>
static cudaError_t launch_f32(const StepArgs &a, int block, cudaStream_t st) {
  if (a.p.n == 0) return cudaSuccess;
  switch (geo_of(a.g)) {
    case GEO_FLAT: return launch_geo<Store, GEO_FLAT>(a, block, st);
    case GEO_SPH: return launch_geo<Store, GEO_SPH>(a, block, st);
    default: return launch_geo<Store, GEO_SPH_PER>(a, block, st);
  }
}

cudaError_t launch_advect_plain(const StepArgs &a, int real, int storage, int block,
                                cudaStream_t st) {
  if (real == PG_POS_F64) return launch_advect_f64(a, storage, block, st);
  if ((a.k.beh & (BEH_SETTLE | BEH_AGE | BEH_SAMPLE)) || a.f.nearest || a.k.scheme == 2)
    return storage == PG_F32 ? launch_advect_plain_ext(a, block, st) : cudaErrorNotSupported;
  switch (storage) {
    case PG_F32: return launch_f32<float>(a, block, st);
    case PG_F16S: return launch_f32<__half>(a, block, st);
    case PG_BF16S: return launch_f32<__nv_bfloat16>(a, block, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace pg
