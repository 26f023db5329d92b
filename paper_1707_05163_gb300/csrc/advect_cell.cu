// advect_cell.cu -- instantiations of the cell-index + offset advection chunk
// (FP32 offsets; FP32, FP16 or BF16 field storage) and the conversions
// between physical positions and the cell form.
#include "advect_cell.cuh"
#include "pg_host.h"

namespace pg {

template <typename Store, int GEO>
static cudaError_t launch_geo(const StepArgs &a, int block, cudaStream_t st) {
  if (a.f.nf == 3) return launch_clamped<advect_cell_kernel<Store, 3, true, GEO>>(a, block, st);
  if (a.g.nz > 1) return launch_clamped<advect_cell_kernel<Store, 2, true, GEO>>(a, block, st);
  return launch_clamped<advect_cell_kernel<Store, 2, false, GEO>>(a, block, st);
}

template <typename Store>
static cudaError_t launch_cell(const StepArgs &a, int block, cudaStream_t st) {
  if (a.p.n == 0) return cudaSuccess;
  switch (geo_of(a.g)) {
    case GEO_FLAT: return launch_geo<Store, GEO_FLAT>(a, block, st);
    case GEO_SPH: return launch_geo<Store, GEO_SPH>(a, block, st);
    default: return launch_geo<Store, GEO_SPH_PER>(a, block, st);
  }
}

cudaError_t launch_advect_cell(const StepArgs &a, int storage, int block, cudaStream_t st) {
  switch (storage) {
    case PG_F32: return launch_cell<float>(a, block, st);
    case PG_F16S: return launch_cell<__half>(a, block, st);
    case PG_BF16S: return launch_cell<__nv_bfloat16>(a, block, st);
    default: return cudaErrorInvalidValue;
  }
}

namespace {

// index coordinate u = (p - x0) / dx in FP64, split into cell and offset
__device__ __forceinline__ void to_cell(double p, double x0, double d, int n, bool periodic,
                                        int &i, float &f) {
  if (periodic) {
    double r = fmod(p - x0, 360.0);
    if (r < 0.0) r += 360.0;
    p = x0 + r;
  }
  const double u = (p - x0) / d;
  double fl = floor(u);
  const double lim = periodic ? (double)(n - 1) : (double)(n - 2);
  if (fl < 0.0) fl = 0.0;
  if (fl > lim) fl = lim;
  i = (int)fl;
  f = (float)(u - fl);
  if (f >= 1.0f && (periodic || i < n - 2)) {   // rounded up to the next node
    f = 0.0f;
    i = i + 1 == n ? 0 : i + 1;
  }
}

__global__ void to_cell_kernel(GridArgs g, const double *lon, const double *lat,
                               const double *dep, int32_t *ci, int32_t *cj, int32_t *ck,
                               float *fx, float *fy, float *fz, int64_t n) {
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n;
       p += (int64_t)gridDim.x * blockDim.x) {
    int i, j, k = 0;
    float x, y, z = 0.f;
    to_cell(lon[p], g.x0[0], g.d[0], g.nx, g.periodic, i, x);
    to_cell(lat[p], g.x0[1], g.d[1], g.ny, false, j, y);
    if (g.nz > 1) to_cell(dep ? dep[p] : g.x0[2], g.x0[2], g.d[2], g.nz, false, k, z);
    ci[p] = i; cj[p] = j; ck[p] = k; fx[p] = x; fy[p] = y; fz[p] = z;
  }
}

__global__ void from_cell_kernel(GridArgs g, const int32_t *ci, const int32_t *cj,
                                 const int32_t *ck, const float *fx, const float *fy,
                                 const float *fz, double *lon, double *lat, double *dep,
                                 int64_t n) {
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n;
       p += (int64_t)gridDim.x * blockDim.x) {
    // x0 + (i + f) d with one rounding of the product-sum (fused multiply-add)
    if (lon) lon[p] = __fma_rn((double)ci[p] + (double)fx[p], g.d[0], g.x0[0]);
    if (lat) lat[p] = __fma_rn((double)cj[p] + (double)fy[p], g.d[1], g.x0[1]);
    if (dep) dep[p] = g.nz > 1 ? __fma_rn((double)ck[p] + (double)fz[p], g.d[2], g.x0[2]) : 0.0;
  }
}

int grid_n(int64_t n, int sm) {
  int64_t g = (n + 255) / 256;
  if (g > (int64_t)sm * 16) g = (int64_t)sm * 16;
  return (int)(g < 1 ? 1 : g);
}

}  // namespace

cudaError_t launch_to_cell(const GridArgs &g, const double *lon, const double *lat,
                           const double *dep, int32_t *ci, int32_t *cj, int32_t *ck, float *fx,
                           float *fy, float *fz, int64_t n, int sm, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  to_cell_kernel<<<grid_n(n, sm), 256, 0, st>>>(g, lon, lat, dep, ci, cj, ck, fx, fy, fz, n);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_from_cell(const GridArgs &g, const int32_t *ci, const int32_t *cj,
                             const int32_t *ck, const float *fx, const float *fy, const float *fz,
                             double *lon, double *lat, double *dep, int64_t n, int sm,
                             cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  from_cell_kernel<<<grid_n(n, sm), 256, 0, st>>>(g, ci, cj, ck, fx, fy, fz, lon, lat, dep, n);
  note_launches(1);
  return cudaGetLastError();
}

}  // namespace pg
