// advect_f64.cu -- FP64 instantiations of the plain advection chunk.
// Compiled with -fmad=false: every multiply and add rounds separately, in the
// order the source states, as in the FP64 definition of the step.
#include "advect_plain.cuh"
#include "pg_host.h"

namespace pg {

template <typename Store>
static cudaError_t launch_f64(const StepArgs &a, int block, cudaStream_t st) {
  if (a.p.n == 0) return cudaSuccess;
  if (a.f.nf == 3)
    return launch_clamped<advect_plain_kernel<double, Store, 3, true, GEO_ANY>>(a, block, st);
  if (a.g.nz > 1)
    return launch_clamped<advect_plain_kernel<double, Store, 2, true, GEO_ANY>>(a, block, st);
  return launch_clamped<advect_plain_kernel<double, Store, 2, false, GEO_ANY>>(a, block, st);
}

cudaError_t launch_advect_f64(const StepArgs &a, int storage, int block, cudaStream_t st) {
  if (storage == PG_F64) return launch_f64<double>(a, block, st);
  if (storage == PG_F32) return launch_f64<float>(a, block, st);
  return cudaErrorInvalidValue;
}

}  // namespace pg
