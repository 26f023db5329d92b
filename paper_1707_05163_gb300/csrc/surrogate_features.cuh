// surrogate_features.cuh -- the learned flow map's per-particle input and
// output, shared by the separate feature and apply kernels (surrogate.cu)
// and by the fused network step (mlp_fused.cu), so both compute the same
// bits.
//
// Features of a particle at time t (37 floats):
//   0 xi, 1 eta       position inside its lon / lat cell, in [0, 1]
//   2 lat / 90, 3 depth / 1000 m, 4 phase of the field's period in [0, 1)
//   5..36             U and V / 0.3 m/s at the 4 x 4 nodes around the cell
//                     (i-1..i+2, j-1..j+2), interpolated linearly in depth
//                     and in time to the particle's depth and time
// Output (3 floats): displacement over the horizon in cells of lon and lat,
// and in units of 100 m of depth.
#pragma once

#include "advect_common.cuh"

namespace pg {

constexpr int kSurFeat = 37;
constexpr float kSurVelScale = 1.0f / 0.3f;
constexpr float kSurDepthUnit = 100.0f;

// Linear interpolation a + (b - a) w with one rounding per operation (the
// same in every kernel that inlines it).
__device__ __forceinline__ float sur_lerp(float a, float b, float w) {
  return __fadd_rn(a, __fmul_rn(__fsub_rn(b, a), w));
}

// The 37 features of an alive particle (FP32 storage, interleaved U/V(/W)
// slabs).  Returns 0, or a device error code (time outside the field, a
// snapshot not resident) with o untouched.
__device__ __forceinline__ int surrogate_features(const GridArgs &g, const FieldArgs &f,
                                                  float lon, float lat, float dep, double time,
                                                  float (&o)[kSurFeat]) {
  // cell and fractions
  const float q = wrap_lon(lon, g.lonf[0]);
  int i;
  float xi;
  if (q >= g.lonf[g.nx - 1]) {
    i = g.nx - 1;
    xi = __fdiv_rn(__fsub_rn(q, g.lonf[g.nx - 1]), __fsub_rn(g.lon_end_f, g.lonf[g.nx - 1]));
  } else {
    i = axis_search<float>(g, 0, g.nx, q);
    xi = __fdiv_rn(__fsub_rn(q, g.lonf[i]), __fsub_rn(g.lonf[i + 1], g.lonf[i]));
  }
  const float y = fminf(fmaxf(lat, g.latf[0]), g.latf[g.ny - 1]);
  const int j = axis_search<float>(g, 1, g.ny, y);
  const float eta = __fdiv_rn(__fsub_rn(y, g.latf[j]), __fsub_rn(g.latf[j + 1], g.latf[j]));
  int k = 0;
  float zeta = 0.f;
  if (g.nz > 1) {
    const float z = fminf(fmaxf(dep, g.depthf[0]), g.depthf[g.nz - 1]);
    k = axis_search<float>(g, 2, g.nz, z);
    zeta = __fdiv_rn(__fsub_rn(z, g.depthf[k]), __fsub_rn(g.depthf[k + 1], g.depthf[k]));
  }
  // time interval
  int s0 = 0, s1 = 0;
  float tau = 0.f, phase = 0.f;
  if (f.nt > 1) {
    double tt, ta, tb;
    int a0 = -1, a1 = -1;
    if (!time_interval(f, time, a0, a1, tt, ta, tb)) return (int)DEVERR_TIME_RANGE;
    s0 = a0; s1 = a1;
    tau = (float)((tt - ta) / (tb - ta));
    if (f.period > 0.0) phase = (float)((tt - f.times[0]) / f.period);
  }
  const float *S0 = reinterpret_cast<const float *>(f.tab[s0]);
  const float *S1 = reinterpret_cast<const float *>(f.tab[s1]);
  if (!S0 || !S1) return (int)DEVERR_SLAB_MISSING;
  const int stride = f.nf == 2 ? 2 : 4;
  o[0] = xi; o[1] = eta;
  o[2] = __fmul_rn(lat, 1.0f / 90.0f);
  o[3] = __fmul_rn(dep, 1e-3f);
  o[4] = phase;
  const size_t level = g.nz > 1 ? (size_t)g.ny * g.nx * stride : 0;
#pragma unroll
  for (int dj = -1; dj <= 2; ++dj) {
    const int jj = min(max(j + dj, 0), g.ny - 1);
#pragma unroll
    for (int di = -1; di <= 2; ++di) {
      int ii = i + di;
      if (ii < 0) ii += g.nx;
      if (ii >= g.nx) ii -= g.nx;
      // U and V of a node are adjacent in the slab: one 8-byte load per
      // node, level and snapshot
      const size_t n0 = (((size_t)k * g.ny + jj) * g.nx + ii) * stride;
      const float2 a0 = __ldg(reinterpret_cast<const float2 *>(S0 + n0));
      const float2 a1 = __ldg(reinterpret_cast<const float2 *>(S0 + n0 + level));
      const float2 b0 = __ldg(reinterpret_cast<const float2 *>(S1 + n0));
      const float2 b1 = __ldg(reinterpret_cast<const float2 *>(S1 + n0 + level));
      const int q2 = 5 + 2 * ((dj + 1) * 4 + (di + 1));
      const float au = sur_lerp(a0.x, a1.x, zeta), bu = sur_lerp(b0.x, b1.x, zeta);
      const float av = sur_lerp(a0.y, a1.y, zeta), bv = sur_lerp(b0.y, b1.y, zeta);
      o[q2] = __fmul_rn(sur_lerp(au, bu, tau), kSurVelScale);
      o[q2 + 1] = __fmul_rn(sur_lerp(av, bv, tau), kSurVelScale);
    }
  }
  return 0;
}

// Apply a predicted displacement (y0, y1: cells of lon and lat; y2: 100 m of
// depth) to an alive particle.  Returns 0 with the position updated, or the
// status of a particle that left the domain (1 lon/lat, 2 depth, 3 NaN) with
// the position untouched.
__device__ __forceinline__ uint8_t surrogate_apply(const GridArgs &g, float &lon, float &lat,
                                                   float &dep, float y0, float y1, float y2) {
  float nl = __fadd_rn(lon, __fmul_rn(y0, g.df[0]));
  const float na = __fadd_rn(lat, __fmul_rn(y1, g.df[1]));
  const float nd = __fadd_rn(dep, __fmul_rn(y2, kSurDepthUnit));
  if (g.periodic) nl = wrap_lon(nl, g.lonf[0]);
  uint8_t st = 0;
  if (!g.periodic && !(nl >= g.lonf[0] && nl <= g.lonf[g.nx - 1])) st = 1;
  else if (!(na >= g.latf[0] && na <= g.latf[g.ny - 1])) st = 1;
  else if (g.nz > 1 && !(nd >= g.depthf[0] && nd <= g.depthf[g.nz - 1])) st = 2;
  else if (!(nl == nl)) st = 3;
  if (st) return st;
  lon = nl; lat = na; dep = nd;
  return 0;
}

}  // namespace pg
