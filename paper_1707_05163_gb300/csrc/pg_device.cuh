// pg_device.cuh -- argument blocks shared by the host side and the kernels,
// plus the device-side counter-based random numbers.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace pg {

// Device-side internal error codes (written once into StepArgs::err).
enum DevErr : int {
  DEVERR_NONE = 0,
  DEVERR_SLAB_MISSING = 1,   // a kernel needed a snapshot that is not resident
  DEVERR_TIME_RANGE = 2,     // a stage time fell outside a non-periodic field
  DEVERR_CELL_INDEX = 3,     // a corner gather was asked for a cell outside the grid
};

struct GridArgs {
  int nx, ny, nz;
  int mesh;                  // 0 flat, 1 spherical
  int periodic;              // zonal wrap
  const double *lon, *lat, *depth;      // FP64 axes (device)
  const float *lonf, *latf, *depthf;    // FP32 copies of the axes (device)
  int uni[3];                // 1 if the axis is uniformly spaced
  double x0[3], inv_d[3];    // first node and 1/spacing (uniform axes)
  float x0f[3], inv_df[3];
  double lon_end;            // lon[0] + 360 (periodic wrap-cell far edge)
  float lon_end_f;
  double lo[3], hi[3];       // first and last node of each axis (kernel
  float lof[3], hif[3];      // parameters, so range tests load nothing)
  // uniform axes, cell form: spacing, and metres -> cells factors (lon on a
  // sphere: 1 / (D dlon), still to be divided by cos(lat))
  double d[3];
  float df[3];
  float inv_m[3];
};

struct FieldArgs {
  int nt;                    // number of snapshots (1 = steady)
  int nf;                    // 2 or 3 fields
  const double *times;       // [nt] (device)
  double period;             // > 0: time-periodic
  const void *const *tab;    // [nt] device pointers to interleaved slabs (null if absent)
  const float *scales;       // [nt * nf] FP32 scales (quantised storage) or null
  int nearest = 0;           // velocities: 0 linear, 1 nearest node in space
  int ntr = 0;               // scalar fields (tracers) sampled into particle variables
  const void *const *ttab = nullptr;   // [ntr * nt] planar tracer slabs (double for FP64
                                       // storage, float otherwise)
  int tnearest[2] = {0, 0};  // per tracer: 0 linear, 1 nearest node
};

struct KernArgs {
  int scheme;                // 0 Euler, 1 RK4
  unsigned beh;              // behaviour bits
  double kh, w_sink;
  uint64_t seed;
  double deg_m;              // metres per degree
  float deg_m_f, inv_deg_m_f, kh_f, w_sink_f;   // FP32 copies for the FP32 path
  double dwell = 0.0, max_age = 0.0;   // settle: dwelling depth (m); age: deletion age (s)
  float dwell_f = 0.f;
  double rk_tol = 0.0, rk_hmin = 0.0, rk_hmax = 0.0;   // RKF45: metres, seconds, seconds
};

// Behaviour bits of the worked example (Sect. 3), beside Brownian (1) and
// sinking (2); and the status of a particle an age behaviour deleted.
enum : unsigned { BEH_SETTLE = 4u, BEH_AGE = 8u, BEH_SAMPLE = 16u };
enum : int { STATUS_DELETED = 4 };

struct PartArgs {
  int64_t n;
  void *x, *y, *z;           // lon, lat, depth (double or float)
  int32_t *ci, *cj, *ck;     // cell form: cell indices
  float *fx, *fy, *fz;       // cell form: offsets in [0, 1)
  double *time;
  const uint64_t *id;
  uint32_t *step;
  uint8_t *status;
  double *age = nullptr;     // [n] seconds of age (age behaviour)
  double *var = nullptr;     // [ntr][vstride] sampled variables (sample behaviour)
  int64_t vstride = 0;
  double *hstep = nullptr;   // [n] RKF45 step lengths (0: start from dt)
};

// Mesh geometry of a kernel instantiation: runtime (GEO_ANY, the FP64 path)
// or fixed at compile time (the FP32 kernels, one instantiation per kind), so
// the per-stage mesh and wrap tests cost nothing.  A periodic zonal boundary
// needs a spherical mesh, so these three kinds cover every field set.
enum : int { GEO_ANY = 0, GEO_FLAT = 1, GEO_SPH = 2, GEO_SPH_PER = 3 };

template <int GEO> __device__ __forceinline__ bool is_sph(const GridArgs &g) {
  if constexpr (GEO == GEO_ANY) return g.mesh == 1;
  else return GEO != GEO_FLAT;
}
template <int GEO> __device__ __forceinline__ bool is_per(const GridArgs &g) {
  if constexpr (GEO == GEO_ANY) return g.periodic != 0;
  else return GEO == GEO_SPH_PER;
}

struct StepArgs {
  GridArgs g;
  FieldArgs f;
  KernArgs k;
  PartArgs p;
  double dt, t_stop, t_end;
  double t_clip;                    // RKF45 steps land on this time (next output) and t_end
  unsigned long long *steps_done;   // particle-steps taken (device counter)
  int *err;                         // first DevErr recorded (device word)
};

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two
// 32x32->64 multiplies mixed with the round key; the key advances by the
// Weyl increments between rounds.  Counter = (id lo, id hi, step, 0), key =
// the particle set's seed.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k.x += 0x9E3779B9u;
      k.y += 0xBB67AE85u;
    }
    const uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
  }
  return c;
}

// 53-bit integers of the two uniforms: u1 = (m1 + 1) 2^-53 in (0, 1],
// u2 = m2 2^-53 in [0, 1).
__device__ __forceinline__ void philox_uniform_bits(uint64_t seed, uint64_t id, uint32_t step,
                                                    unsigned long long &m1,
                                                    unsigned long long &m2) {
  const uint4 r = philox4x32_10(make_uint4((uint32_t)id, (uint32_t)(id >> 32), step, 0u),
                                make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)));
  m1 = ((unsigned long long)(r.x >> 5) << 26) | (unsigned long long)(r.y >> 6);
  m2 = ((unsigned long long)(r.z >> 5) << 26) | (unsigned long long)(r.w >> 6);
}

// Box-Muller in FP64.
__device__ __forceinline__ void normal_pair(uint64_t seed, uint64_t id, uint32_t step,
                                            double &n1, double &n2) {
  unsigned long long m1, m2;
  philox_uniform_bits(seed, id, step, m1, m2);
  const double u1 = ((double)m1 + 1.0) * (1.0 / 9007199254740992.0);
  const double u2 = (double)m2 * (1.0 / 9007199254740992.0);
  const double rad = sqrt(-2.0 * log(u1));
  const double ang = 6.283185307179586 * u2;
  n1 = rad * cos(ang);
  n2 = rad * sin(ang);
}

// Box-Muller in FP32 from the same 53-bit uniforms, each correctly rounded
// to FP32 first (no FP64 arithmetic).
__device__ __forceinline__ void normal_pair(uint64_t seed, uint64_t id, uint32_t step,
                                            float &n1, float &n2) {
  unsigned long long m1, m2;
  philox_uniform_bits(seed, id, step, m1, m2);
  const float u1 = __ull2float_rn(m1 + 1ull) * 1.1102230246251565e-16f;   // 2^-53
  const float u2 = __ull2float_rn(m2) * 1.1102230246251565e-16f;
  const float rad = sqrtf(-2.0f * logf(u1));
  float s, c;
  sincospif(2.0f * u2, &s, &c);
  n1 = rad * c;
  n2 = rad * s;
}

}  // namespace pg
