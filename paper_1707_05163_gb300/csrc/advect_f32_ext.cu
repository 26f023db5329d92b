// advect_f32_ext.cu -- FP32 advection chunk with the worked example's
// behaviours (settle, age, sampled scalar fields; Sect. 3) and
// nearest-neighbour interpolation (Sect. 2.3), on FP32 positions and FP32
// field storage.  A separate instantiation, so the plain FP32 kernels carry
// none of this code.
#include "advect_plain.cuh"
#include "pg_host.h"

namespace pg {

template <int GEO>
static cudaError_t launch_geo_ext(const StepArgs &a, int block, cudaStream_t st) {
  if (a.f.nf == 3)
    return launch_clamped<advect_plain_kernel<float, float, 3, true, GEO, true>>(a, block, st);
  if (a.g.nz > 1)
    return launch_clamped<advect_plain_kernel<float, float, 2, true, GEO, true>>(a, block, st);
  return launch_clamped<advect_plain_kernel<float, float, 2, false, GEO, true>>(a, block, st);
}

cudaError_t launch_advect_plain_ext(const StepArgs &a, int block, cudaStream_t st) {
  if (a.p.n == 0) return cudaSuccess;
  switch (geo_of(a.g)) {
    case GEO_FLAT: return launch_geo_ext<GEO_FLAT>(a, block, st);
    case GEO_SPH: return launch_geo_ext<GEO_SPH>(a, block, st);
    default: return launch_geo_ext<GEO_SPH_PER>(a, block, st);
  }
}

}  // namespace pg
