// mlp_tc.cu -- forward GEMM on the 5th-generation tensor cores (tcgen05).
#include <cuda_bf16.h>

#include "pg_host.h"

namespace pg {

cudaError_t gemm_nt_tc(const __nv_bfloat16 *, int, const __nv_bfloat16 *, int, int64_t, int, int,
                       const float *, int, float *, __nv_bfloat16 *, __nv_bfloat16 *, int,
                       cudaStream_t, int *) {
  return cudaErrorNotSupported;
}

}  // namespace pg
