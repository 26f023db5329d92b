// advect_common.cuh -- pieces shared by the advection kernels: node loads
// of the interleaved field storage, the per-thread cell/snapshot cache
// (Sampler), the snapshot-interval rules, corner gathers and bi/trilinear
// interpolation.
#pragma once

#include "pg_device.cuh"

namespace pg {

// ------------------------------------------------------------ node loads ---
// Interleaved storage: node (k, j, i) holds its NF field values contiguously
// (NF = 3 padded to 4), so one vector load fetches U, V[, W] of a corner.
template <typename Real, int NF>
__device__ __forceinline__ void load_node(const double *p, size_t node, const float *, Real (&v)[NF]) {
  if constexpr (NF == 2) {
    const double2 a = __ldg(reinterpret_cast<const double2 *>(p) + node);
    v[0] = (Real)a.x; v[1] = (Real)a.y;
  } else {
    const double2 a = __ldg(reinterpret_cast<const double2 *>(p) + 2 * node);
    const double2 b = __ldg(reinterpret_cast<const double2 *>(p) + 2 * node + 1);
    v[0] = (Real)a.x; v[1] = (Real)a.y; v[2] = (Real)b.x;
  }
}

template <typename Real, int NF>
__device__ __forceinline__ void load_node(const float *p, size_t node, const float *, Real (&v)[NF]) {
  if constexpr (NF == 2) {
    const float2 a = __ldg(reinterpret_cast<const float2 *>(p) + node);
    v[0] = (Real)a.x; v[1] = (Real)a.y;
  } else {
    const float4 a = __ldg(reinterpret_cast<const float4 *>(p) + node);
    v[0] = (Real)a.x; v[1] = (Real)a.y; v[2] = (Real)a.z;
  }
}

// Quantised storage: value = float(code) * scale, rounded in FP32.
template <typename Real, int NF>
__device__ __forceinline__ void load_node(const __half *p, size_t node, const float *sc, Real (&v)[NF]) {
  if constexpr (NF == 2) {
    const __half2 a = __ldg(reinterpret_cast<const __half2 *>(p) + node);
    v[0] = (Real)(__low2float(a) * sc[0]); v[1] = (Real)(__high2float(a) * sc[1]);
  } else {
    const uint2 a = __ldg(reinterpret_cast<const uint2 *>(p) + node);
    const __half2 lo = *reinterpret_cast<const __half2 *>(&a.x);
    const __half2 hi = *reinterpret_cast<const __half2 *>(&a.y);
    v[0] = (Real)(__low2float(lo) * sc[0]); v[1] = (Real)(__high2float(lo) * sc[1]);
    v[2] = (Real)(__low2float(hi) * sc[2]);
  }
}

template <typename Real, int NF>
__device__ __forceinline__ void load_node(const __nv_bfloat16 *p, size_t node, const float *sc, Real (&v)[NF]) {
  if constexpr (NF == 2) {
    const __nv_bfloat162 a = __ldg(reinterpret_cast<const __nv_bfloat162 *>(p) + node);
    v[0] = (Real)(__low2float(a) * sc[0]); v[1] = (Real)(__high2float(a) * sc[1]);
  } else {
    const uint2 a = __ldg(reinterpret_cast<const uint2 *>(p) + node);
    const __nv_bfloat162 lo = *reinterpret_cast<const __nv_bfloat162 *>(&a.x);
    const __nv_bfloat162 hi = *reinterpret_cast<const __nv_bfloat162 *>(&a.y);
    v[0] = (Real)(__low2float(lo) * sc[0]); v[1] = (Real)(__high2float(lo) * sc[1]);
    v[2] = (Real)(__low2float(hi) * sc[2]);
  }
}

// ------------------------------------------------------- math per Real ---
__device__ __forceinline__ double pg_floor(double a) { return floor(a); }
__device__ __forceinline__ float pg_floor(float a) { return floorf(a); }
__device__ __forceinline__ double pg_sqrt(double a) { return sqrt(a); }
__device__ __forceinline__ float pg_sqrt(float a) { return sqrtf(a); }
__device__ __forceinline__ double pg_fabs(double a) { return fabs(a); }
__device__ __forceinline__ float pg_fabs(float a) { return fabsf(a); }
// cos(lat in degrees)
__device__ __forceinline__ double cos_deg(double lat) {
  const double deg2rad = 3.14159265358979323846 / 180.0;
  return cos(lat * deg2rad);
}
// FP32: the Taylor series of cos x to the x^12 term, x = lat in radians,
// evaluated by Horner's rule in x^2.  On |x| <= pi/2 the remainder is below
// x^14 / 14! < 7e-9; the rounding of x itself dominates (a relative error of
// 7e-7 at 80 degrees, as for any FP32 argument), and there is no range
// reduction or branch.
__device__ __forceinline__ float cos_deg(float lat) {
  const float x = lat * 0.017453292519943295f;
  const float x2 = x * x;
  float p = fmaf(x2, 1.0f / 479001600.0f, -1.0f / 3628800.0f);
  p = fmaf(x2, p, 1.0f / 40320.0f);
  p = fmaf(x2, p, -1.0f / 720.0f);
  p = fmaf(x2, p, 1.0f / 24.0f);
  p = fmaf(x2, p, -0.5f);
  return fmaf(x2, p, 1.0f);
}

// u (m/s) -> degrees/s of longitude at latitude lat; v (m/s) -> degrees/s.
__device__ __forceinline__ double lon_rate(double u, double lat, const KernArgs &k) {
  return u / (k.deg_m * cos_deg(lat));
}
__device__ __forceinline__ float lon_rate(float u, float lat, const KernArgs &k) {
  return __fdividef(u, k.deg_m_f * cos_deg(lat));
}
__device__ __forceinline__ double lat_rate(double v, const KernArgs &k) { return v / k.deg_m; }
__device__ __forceinline__ float lat_rate(float v, const KernArgs &k) { return v * k.inv_deg_m_f; }

template <typename Real> __device__ __forceinline__ const Real *axis(const GridArgs &g, int a);
template <> __device__ __forceinline__ const double *axis<double>(const GridArgs &g, int a) {
  return a == 0 ? g.lon : (a == 1 ? g.lat : g.depth);
}
template <> __device__ __forceinline__ const float *axis<float>(const GridArgs &g, int a) {
  return a == 0 ? g.lonf : (a == 1 ? g.latf : g.depthf);
}
template <typename Real> __device__ __forceinline__ Real axis_x0(const GridArgs &g, int a);
template <> __device__ __forceinline__ double axis_x0<double>(const GridArgs &g, int a) { return g.x0[a]; }
template <> __device__ __forceinline__ float axis_x0<float>(const GridArgs &g, int a) { return g.x0f[a]; }
template <typename Real> __device__ __forceinline__ Real axis_inv(const GridArgs &g, int a);
template <> __device__ __forceinline__ double axis_inv<double>(const GridArgs &g, int a) { return g.inv_d[a]; }
template <> __device__ __forceinline__ float axis_inv<float>(const GridArgs &g, int a) { return g.inv_df[a]; }
__device__ __forceinline__ double axis_lo(const GridArgs &g, int a, double) { return g.lo[a]; }
__device__ __forceinline__ float axis_lo(const GridArgs &g, int a, float) { return g.lof[a]; }
__device__ __forceinline__ double axis_hi(const GridArgs &g, int a, double) { return g.hi[a]; }
__device__ __forceinline__ float axis_hi(const GridArgs &g, int a, float) { return g.hif[a]; }
__device__ __forceinline__ double lon_end(const GridArgs &g, double) { return g.lon_end; }
__device__ __forceinline__ float lon_end(const GridArgs &g, float) { return g.lon_end_f; }

// Full search on one axis: the largest i <= n-2 with x[i] <= p, given that
// x[0] <= p <= x[n-1].  Uniform axes start from floor((p - x0) / dx) and
// correct against the stored nodes; others use bisection.
template <typename Real>
__device__ __forceinline__ int axis_search(const GridArgs &g, int a, int n, Real p) {
  const Real *x = axis<Real>(g, a);
  int i;
  if (g.uni[a]) {
    const Real f = pg_floor((p - axis_x0<Real>(g, a)) * axis_inv<Real>(g, a));
    i = f < (Real)0 ? 0 : (f > (Real)(n - 2) ? n - 2 : (int)f);
    while (i > 0 && x[i] > p) --i;
    while (i < n - 2 && x[i + 1] <= p) ++i;
  } else {
    int lo = 0, hi = n - 1;
    while (hi - lo > 1) {
      const int mid = lo + (hi - lo) / 2;
      if (x[mid] <= p) lo = mid; else hi = mid;
    }
    i = lo;
  }
  return i;
}

// ---------------------------------------------------------- the sampler ---
template <typename Real, typename Store, int NF, bool D3, int GEO = GEO_ANY>
struct Sampler {
  static constexpr int NC = D3 ? 8 : 4;
  // cached cell (ci = -1: none) and its bounds
  int ci, cj, ck;
  Real xlo, xhi, ylo, yhi, zlo, zhi;
  Real rx, ry, rz;            // 1 / (hi - lo), FP32 path only
  // cached snapshot interval and the snapshots whose corners are held
  int s0;                     // first snapshot of the cached pair (second: snap_next)
  // what `v` lacks: 1 the cell changed, 2 the snapshot pair moved on by one
  // (s0 is the old s1), 4 anything else (a new pair, or nothing held yet)
  int dirty;
  double ta;                  // FP32 path: interval start in unwrapped time
  float span, rspan;          // FP32 path
  Real v[2][NF][NC];

  __device__ __forceinline__ void reset() {
    ci = -1; cj = -1; ck = -1; s0 = -1; dirty = 4;
    // empty cells on every axis: the first hit test of each axis fails
    xlo = (Real)1; xhi = (Real)0;
    ylo = (Real)1; yhi = (Real)0;
    zlo = (Real)1; zhi = (Real)0;
  }
};

// Reduce a longitude into [x0, x0 + 360).  FP64: the definition's fmod.
// FP32: stage positions are at most one turn away, so a compare and one
// add/subtract do (fmod for anything farther).
__device__ __forceinline__ double wrap_lon(double p, double x0) {
  double r = fmod(p - x0, 360.0);
  if (r < 0.0) r += 360.0;
  if (r >= 360.0) r -= 360.0;
  return x0 + r;
}
__device__ __forceinline__ float wrap_lon(float p, float x0) {
  float q = p;
  if (q < x0) q += 360.0f;
  else if (q >= x0 + 360.0f) q -= 360.0f;
  if (!(q >= x0 && q < x0 + 360.0f)) {
    float r = fmodf(p - x0, 360.0f);
    if (r < 0.0f) r += 360.0f;
    if (r >= 360.0f) r -= 360.0f;
    q = x0 + r;
  }
  return q;
}

// Is p inside the cached cell [lo, hi]?  FP64: the definition's half-open
// cell, closed only at the last node.  FP32: closed on both sides.
template <typename Real>
__device__ __forceinline__ bool in_cell(Real p, Real lo, Real hi, bool last) {
  if constexpr (sizeof(Real) == 8) return p >= lo && (p < hi || (last && p == hi));
  else return p >= lo && p <= hi;
}

// Snapshot interval for time t in FP64 (the definition's rules: the largest
// s <= nt-2 with T[s] <= t; periodic fields reduce t into [T0, T0 + period)
// and interpolate from the last snapshot to the first after T[nt-1]).
// Writes s0, s1, the wrapped time tt and the interval bounds.
__device__ __forceinline__ bool time_interval(const FieldArgs &f, double t, int &s0, int &s1,
                                              double &tt, double &ta, double &tb) {
  const double *T = f.times;
  const int nt = f.nt;
  tt = t;
  if (f.period > 0.0) {
    double r = t - T[0];
    if (!(r >= 0.0 && r < f.period)) {   // fmod is the identity on [0, period)
      r = fmod(r, f.period);
      if (r < 0.0) r += f.period;
    }
    tt = T[0] + r;
    if (tt >= T[nt - 1]) {
      s0 = nt - 1; s1 = 0;
      ta = T[nt - 1]; tb = T[0] + f.period;
      return true;
    }
  }
  if (!(tt >= T[0] && tt <= T[nt - 1])) return false;
  int lo = 0, hi = nt - 1;
  if (s0 >= 0 && s0 <= nt - 2 && T[s0] <= tt && (tt < T[s0 + 1] || (s0 == nt - 2 && tt == T[nt - 1]))) {
    lo = s0;
  } else {
    while (hi - lo > 1) {
      const int mid = lo + (hi - lo) / 2;
      if (T[mid] <= tt) lo = mid; else hi = mid;
    }
  }
  s0 = lo; s1 = lo + 1;
  ta = T[lo]; tb = T[lo + 1];
  return true;
}

// Second snapshot of the pair that starts at s0: s0 + 1, or the first
// snapshot after the last one (periodic fields; a steady field's pair is
// (0, 0)).  These are the only pairs time_interval returns.
__device__ __forceinline__ int snap_next(const FieldArgs &f, int s0) {
  return s0 + 1 < f.nt ? s0 + 1 : 0;
}

template <typename Real, typename Store, int NF, bool D3, int GEO, class A>
__device__ __forceinline__ bool gather_slab(const A &a, Sampler<Real, Store, NF, D3, GEO> &c,
                                            int sl, int s) {
  const GridArgs &g = a.g;
  const Store *base = reinterpret_cast<const Store *>(a.f.tab[s]);
  if (base == nullptr) {
    atomicCAS(a.err, 0, (int)DEVERR_SLAB_MISSING);
    return false;
  }
  // the cached cell must be a cell of the grid (the periodic wrap cell is
  // nx-1, joining node nx-1 to node 0); anything else is an internal error
  // recorded in a.err, never a read outside the slab
  if (!((unsigned)c.ci < (unsigned)g.nx && (unsigned)c.cj <= (unsigned)(g.ny - 2) &&
        (!D3 || (unsigned)c.ck <= (unsigned)(g.nz - 2)) && (D3 || c.ck == 0))) {
    atomicCAS(a.err, 0, (int)DEVERR_CELL_INDEX);
    return false;
  }
  const int ci1 = c.ci + 1 == g.nx ? 0 : c.ci + 1;   // the periodic wrap cell joins nx-1 to 0
  float sc[3] = {1.f, 1.f, 1.f};
  if (a.f.scales != nullptr) {
#pragma unroll
    for (int f = 0; f < NF; ++f) sc[f] = a.f.scales[s * NF + f];
  }
#pragma unroll
  for (int kk = 0; kk < (D3 ? 2 : 1); ++kk) {
#pragma unroll
    for (int jj = 0; jj < 2; ++jj) {
      const size_t row = ((size_t)(c.ck + kk) * g.ny + (size_t)(c.cj + jj)) * g.nx;
#pragma unroll
      for (int ii = 0; ii < 2; ++ii) {
        Real vv[NF];
        load_node<Real, NF>(base, row + (size_t)(ii ? ci1 : c.ci), sc, vv);
#pragma unroll
        for (int f = 0; f < NF; ++f) c.v[sl][f][kk * 4 + jj * 2 + ii] = vv[f];
      }
    }
  }
  return true;
}

// Make `v` hold the corners of the cached cell for snapshots s0 and s1.  If
// only the snapshot pair moved on by one, the shared snapshot's corners move
// from slot 1 to slot 0 and only the new snapshot is read.
template <typename Real, typename Store, int NF, bool D3, int GEO, class A>
__device__ __forceinline__ bool gather(const A &a, Sampler<Real, Store, NF, D3, GEO> &c,
                                       bool steady) {
  if (steady) {
    if (!gather_slab(a, c, 0, c.s0)) return false;
    if constexpr (sizeof(Real) == 4) {     // FP32 interpolates both slots
#pragma unroll
      for (int f = 0; f < NF; ++f)
#pragma unroll
        for (int q = 0; q < Sampler<Real, Store, NF, D3, GEO>::NC; ++q) c.v[1][f][q] = c.v[0][f][q];
    }
  } else if (c.dirty == 2) {
#pragma unroll
    for (int f = 0; f < NF; ++f)
#pragma unroll
      for (int q = 0; q < Sampler<Real, Store, NF, D3, GEO>::NC; ++q) c.v[0][f][q] = c.v[1][f][q];
    if (!gather_slab(a, c, 1, snap_next(a.f, c.s0))) return false;
  } else {
    if (!gather_slab(a, c, 0, c.s0)) return false;
    if (!gather_slab(a, c, 1, snap_next(a.f, c.s0))) return false;
  }
  c.dirty = 0;
  return true;
}

// FP64 spatial interpolation in the definition's order: bilinear weights
// applied as (w00 f00 + w10 f10) + (w11 f11 + w01 f01); trilinear is linear in
// zeta between the two levels.
template <typename Real, int NC>
__device__ __forceinline__ Real interp_space(const Real (&v)[NC], Real xi, Real eta, Real zeta) {
  const Real w00 = ((Real)1 - xi) * ((Real)1 - eta);
  const Real w10 = xi * ((Real)1 - eta);
  const Real w11 = xi * eta;
  const Real w01 = ((Real)1 - xi) * eta;
  const Real a = (w00 * v[0] + w10 * v[1]) + (w11 * v[3] + w01 * v[2]);
  if constexpr (NC == 4) {
    return a;
  } else {
    const Real b = (w00 * v[4] + w10 * v[5]) + (w11 * v[7] + w01 * v[6]);
    return ((Real)1 - zeta) * a + zeta * b;
  }
}

// Time of the current step.  FP64 path: `t` is the exact step start.  FP32
// path: the step start is t + k * dt, known to the kernel only as `d`, its
// FP32 offset inside the cached snapshot interval; the FP64 value is formed
// only when a stage leaves that interval.
struct Clock {
  double t, dt;
  int k;
  float d;
  bool tin = false;          // FP32: the current step lies in the cached interval
  __device__ __forceinline__ double start() const { return t + (double)k * dt; }
};

template <typename Real, int GEO>
__device__ __forceinline__ int out_of_domain(const GridArgs &g, Real lon, Real lat, Real dep,
                                             bool d3) {
  const Real z = (Real)0;
  if (!is_per<GEO>(g) && !(lon >= axis_lo(g, 0, z) && lon <= axis_hi(g, 0, z))) return 1;
  if (is_per<GEO>(g) && !(lon == lon)) return 1;
  if (!(lat >= axis_lo(g, 1, z) && lat <= axis_hi(g, 1, z))) return 1;
  if (d3 && !(dep >= axis_lo(g, 2, z) && dep <= axis_hi(g, 2, z))) return 2;
  return 0;
}

__device__ __forceinline__ double kh_of(const KernArgs &k, double) { return k.kh; }
__device__ __forceinline__ float kh_of(const KernArgs &k, float) { return k.kh_f; }
__device__ __forceinline__ double w_of(const KernArgs &k, double) { return k.w_sink; }
__device__ __forceinline__ float w_of(const KernArgs &k, float) { return k.w_sink_f; }

// FP32: bring the snapshot interval of the stage time (step start + off)
// and the corner cache up to date -- the slow part of a stage, skipped while
// the stage stays in the cached cell and interval.  The stage time is an
// FP32 offset inside the cached interval; the FP64 step start is formed only
// when a stage leaves it.  Returns 0, or -1 for an internal failure recorded
// in a.err.
template <typename Store, int NF, bool D3, int GEO, class A>
__device__ __forceinline__ int refresh32(const A &a, Sampler<float, Store, NF, D3, GEO> &c,
                                         Clock &ck, float off) {
  const bool steady = a.f.nt == 1;
  if (!steady) {
    const float d = ck.d + off;
    if (!(c.s0 >= 0 && d >= 0.f && d <= c.span)) {
      const double t0 = ck.start();
      const double ts = t0 + (double)off;
      double tt, ta, tb;
      int s0 = c.s0, s1 = snap_next(a.f, c.s0);
      if (!time_interval(a.f, ts, s0, s1, tt, ta, tb)) {
        atomicCAS(a.err, 0, (int)DEVERR_TIME_RANGE);
        return -1;
      }
      if (s0 != c.s0) c.dirty |= (c.s0 >= 0 && s0 == snap_next(a.f, c.s0)) ? 2 : 4;
      c.s0 = s0;
      c.ta = ts - (tt - ta);              // interval start in unwrapped time
      c.span = (float)(tb - ta);
      c.rspan = 1.0f / c.span;
      ck.d = (float)(t0 - c.ta);
    }
  } else {
    c.s0 = 0;
  }
  if (c.dirty) {
    if (!gather(a, c, steady)) return -1;
  }
  return 0;
}

// FP32 time weight of the stage inside the cached interval (0 for a steady
// field).
template <typename Store, int NF, bool D3, int GEO, class A>
__device__ __forceinline__ float tau32(const A &a, const Sampler<float, Store, NF, D3, GEO> &c,
                                       const Clock &ck, float off) {
  return a.f.nt == 1 ? 0.f : fminf((ck.d + off) * c.rspan, 1.0f);
}

// FP32 spatial interpolation as one weighted sum over the corners, the
// weights formed once per stage (bilinear, or trilinear as the bilinear
// weights times 1 - zeta and zeta).  The sum runs in corner order (i, j),
// (i+1, j), (i, j+1), (i+1, j+1)[, the same on level k+1] as one chain of
// fused multiply-adds; on a cell face the weights of the far corners are
// exactly 0 and the remaining terms come in the same order from either
// neighbouring cell, so the two cells give the same value there.
template <int NC>
__device__ __forceinline__ void corner_weights(float xi, float eta, float zeta, float (&w)[NC]) {
  const float x0 = 1.f - xi, y0 = 1.f - eta;
  const float w00 = x0 * y0, w10 = xi * y0, w01 = x0 * eta, w11 = xi * eta;
  if constexpr (NC == 4) {
    w[0] = w00; w[1] = w10; w[2] = w01; w[3] = w11;
  } else {
    const float z0 = 1.f - zeta;
    w[0] = w00 * z0; w[1] = w10 * z0; w[2] = w01 * z0; w[3] = w11 * z0;
    w[4] = w00 * zeta; w[5] = w10 * zeta; w[6] = w01 * zeta; w[7] = w11 * zeta;
  }
}

template <int NC>
__device__ __forceinline__ float weighted_sum(const float (&v)[NC], const float (&w)[NC]) {
  float acc = w[0] * v[0];
#pragma unroll
  for (int q = 1; q < NC; ++q) acc = fmaf(w[q], v[q], acc);
  return acc;
}

// Nearest-neighbour pick among the corners of the cached cell: corner index
// (i + 1 if xi > 1/2) + 2 (j + 1 if eta > 1/2) + 4 (k + 1 if zeta > 1/2), the
// lower node on a tie.  A select chain, so a NaN at another corner does not
// reach the result.
template <int NC, typename Real>
__device__ __forceinline__ Real pick_corner(const Real (&v)[NC], int qi) {
  Real r = v[0];
#pragma unroll
  for (int q = 1; q < NC; ++q) r = (qi == q) ? v[q] : r;
  return r;
}

template <typename Real>
__device__ __forceinline__ int nearest_corner(Real xi, Real eta, Real zeta) {
  return (xi > (Real)0.5 ? 1 : 0) | (eta > (Real)0.5 ? 2 : 0) | (zeta > (Real)0.5 ? 4 : 0);
}

// FP32 field values from the cached corners: spatial interpolation in both
// snapshots (weighted_sum), then (1 - tau) a + tau b, exact at both ends, so a stage time on
// a snapshot gives the same value from either neighbouring interval (results
// do not depend on which interval a thread has cached).  A steady field holds
// its snapshot in both slots with tau = 0, which returns a exactly, so there
// is no branch on steadiness.  One NaN test per stage covers all components
// (same outcome as a test per value: PG_NAN, state untouched) and leaves the
// interpolations free of branches; CHECK = false leaves the test to the
// caller.  Returns 0 or PG_NAN (3).
template <typename Store, int NF, bool D3, int GEO, bool CHECK = true>
__device__ __forceinline__ int interp32(const Sampler<float, Store, NF, D3, GEO> &c, float xi,
                                        float eta, float zeta, float tau, float (&vel)[3]) {
  constexpr int NC = Sampler<float, Store, NF, D3, GEO>::NC;
  float w[NC];
  corner_weights<NC>(xi, eta, zeta, w);
#pragma unroll
  for (int f = 0; f < NF; ++f) {
    const float va = weighted_sum<NC>(c.v[0][f], w);
    const float vb = weighted_sum<NC>(c.v[1][f], w);
    vel[f] = fmaf(tau, vb, (1.0f - tau) * va);
  }
  if constexpr (NF == 2) vel[2] = 0.f;
  if (CHECK && (!(vel[0] == vel[0]) | !(vel[1] == vel[1]) | !(vel[2] == vel[2]))) return 3;
  return 0;
}

// FP32 nearest-neighbour values: the nearest corner in each snapshot, then
// (1 - tau) a + tau b.
template <typename Store, int NF, bool D3, int GEO>
__device__ __forceinline__ void nearest32(const Sampler<float, Store, NF, D3, GEO> &c, float xi,
                                          float eta, float zeta, float tau, float (&vel)[3]) {
  constexpr int NC = Sampler<float, Store, NF, D3, GEO>::NC;
  const int qi = nearest_corner(xi, eta, D3 ? zeta : 0.f);
#pragma unroll
  for (int f = 0; f < NF; ++f) {
    const float va = pick_corner<NC>(c.v[0][f], qi);
    const float vb = pick_corner<NC>(c.v[1][f], qi);
    vel[f] = fmaf(tau, vb, (1.0f - tau) * va);
  }
  if constexpr (NF == 2) vel[2] = 0.f;
}

// Field values (m/s) at a stage, once the cell (c.ci, c.cj, c.ck) and the
// fractions (xi, eta, zeta) are known: snapshot interval of the stage time
// (step start + off), corner gather if the cell or interval changed, spatial
// interpolation in each snapshot, then linear interpolation in time.
// Returns 0, PG_NAN (3), or -1 for an internal failure recorded in a.err.
template <typename Real, typename Store, int NF, bool D3, int GEO, class A>
__device__ __forceinline__ int sample_fields(const A &a, Sampler<Real, Store, NF, D3, GEO> &c,
                                             Clock &ck, Real off, Real xi, Real eta, Real zeta,
                                             Real (&vel)[3]) {
  if constexpr (sizeof(Real) == 4) {
    if (refresh32(a, c, ck, off)) return -1;
    return interp32(c, xi, eta, zeta, tau32(a, c, ck, off), vel);
  } else {
    // FP64: the definition -- interval and a + (b - a) tau for every stage,
    // and its NaN test per value
    const bool steady = a.f.nt == 1;
    Real tau = (Real)0;
    if (!steady) {
      const double ts = ck.t + (double)off;
      double tt, ta, tb;
      int s0 = c.s0, s1 = snap_next(a.f, c.s0);
      if (!time_interval(a.f, ts, s0, s1, tt, ta, tb)) {
        atomicCAS(a.err, 0, (int)DEVERR_TIME_RANGE);
        return -1;
      }
      if (s0 != c.s0) c.dirty |= (c.s0 >= 0 && s0 == snap_next(a.f, c.s0)) ? 2 : 4;
      c.s0 = s0;
      tau = (tt - ta) / (tb - ta);
    } else {
      c.s0 = 0;
    }
    if (c.dirty) {
      if (!gather(a, c, steady)) return -1;
    }
    constexpr int NC = Sampler<Real, Store, NF, D3, GEO>::NC;
    const int qi = nearest_corner(xi, eta, D3 ? zeta : (Real)0);
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      Real val = a.f.nearest ? pick_corner<NC>(c.v[0][f], qi)
                             : interp_space<Real, NC>(c.v[0][f], xi, eta, zeta);
      if (!steady) {
        const Real b = a.f.nearest ? pick_corner<NC>(c.v[1][f], qi)
                                   : interp_space<Real, NC>(c.v[1][f], xi, eta, zeta);
        val = val + (b - val) * tau;
      }
      if (!(val == val)) return 3;
      vel[f] = val;
    }
    if constexpr (NF == 2) vel[2] = (Real)0;
    return 0;
  }
}

// ------------------------------------------------------ scalar fields ---
// Value of scalar field q (a tracer such as temperature, Sect. 3) at a
// position and time, in FP64 with every product and sum rounded separately
// (no fused multiply-add, in the order of the definition): the cell on each
// axis by a full search, the wrap cell on a periodic zonal axis, bilinear
// weights applied as (w00 f00 + w10 f10) + (w11 f11 + w01 f01), linear in
// depth between two levels, or the nearest node; linear in time.  Positions
// are inside the domain when this is called.  Returns false (and records an
// internal error) when a snapshot is missing or the time is outside a
// non-periodic field.
template <typename TS>
__device__ __forceinline__ double tracer_node(const TS *b, const GridArgs &g, int k, int j, int i) {
  return (double)b[((size_t)k * g.ny + (size_t)j) * g.nx + (size_t)i];
}

__device__ __forceinline__ double lerp_rn(double a, double b, double w) {
  return __dadd_rn(a, __dmul_rn(__dadd_rn(b, -a), w));      // a + (b - a) w
}

template <typename TS>
__device__ __noinline__ bool tracer_value(const GridArgs &g, const FieldArgs &f, int q, double lon,
                                          double lat, double dep, double t, double &out, int *err) {
  int i0, i1;
  double xi;
  if (g.periodic) {
    const double p = wrap_lon(lon, g.lon[0]);
    if (p >= g.lon[g.nx - 1]) {
      i0 = g.nx - 1; i1 = 0;
      xi = __ddiv_rn(__dadd_rn(p, -g.lon[g.nx - 1]), __dadd_rn(g.lon_end, -g.lon[g.nx - 1]));
    } else {
      i0 = axis_search<double>(g, 0, g.nx, p); i1 = i0 + 1;
      xi = __ddiv_rn(__dadd_rn(p, -g.lon[i0]), __dadd_rn(g.lon[i1], -g.lon[i0]));
    }
  } else {
    i0 = axis_search<double>(g, 0, g.nx, lon); i1 = i0 + 1;
    xi = __ddiv_rn(__dadd_rn(lon, -g.lon[i0]), __dadd_rn(g.lon[i1], -g.lon[i0]));
  }
  const int j0 = axis_search<double>(g, 1, g.ny, lat), j1 = j0 + 1;
  const double eta = __ddiv_rn(__dadd_rn(lat, -g.lat[j0]), __dadd_rn(g.lat[j1], -g.lat[j0]));
  int k0 = 0, k1 = 0;
  double zeta = 0.0;
  if (g.nz > 1) {
    k0 = axis_search<double>(g, 2, g.nz, dep); k1 = k0 + 1;
    zeta = __ddiv_rn(__dadd_rn(dep, -g.depth[k0]), __dadd_rn(g.depth[k1], -g.depth[k0]));
  }
  int s0 = 0, s1 = 0;
  double tau = 0.0;
  if (f.nt > 1) {
    double tt, ta, tb;
    s0 = -1;
    if (!time_interval(f, t, s0, s1, tt, ta, tb)) {
      atomicCAS(err, 0, (int)DEVERR_TIME_RANGE);
      return false;
    }
    tau = __ddiv_rn(__dadd_rn(tt, -ta), __dadd_rn(tb, -ta));
  }
  double val[2] = {0.0, 0.0};
  for (int r = 0; r < (f.nt > 1 ? 2 : 1); ++r) {
    const TS *b = reinterpret_cast<const TS *>(f.ttab[q * f.nt + (r == 0 ? s0 : s1)]);
    if (b == nullptr) {
      atomicCAS(err, 0, (int)DEVERR_SLAB_MISSING);
      return false;
    }
    if (f.tnearest[q]) {
      val[r] = tracer_node(b, g, zeta > 0.5 ? k1 : k0, eta > 0.5 ? j1 : j0, xi > 0.5 ? i1 : i0);
    } else {
      const double w00 = __dmul_rn(__dadd_rn(1.0, -xi), __dadd_rn(1.0, -eta));
      const double w10 = __dmul_rn(xi, __dadd_rn(1.0, -eta));
      const double w11 = __dmul_rn(xi, eta);
      const double w01 = __dmul_rn(__dadd_rn(1.0, -xi), eta);
      double lev[2] = {0.0, 0.0};
      for (int kk = 0; kk < (g.nz > 1 ? 2 : 1); ++kk) {
        const int k = kk ? k1 : k0;
        lev[kk] = __dadd_rn(__dadd_rn(__dmul_rn(w00, tracer_node(b, g, k, j0, i0)),
                                      __dmul_rn(w10, tracer_node(b, g, k, j0, i1))),
                            __dadd_rn(__dmul_rn(w11, tracer_node(b, g, k, j1, i1)),
                                      __dmul_rn(w01, tracer_node(b, g, k, j1, i0))));
      }
      val[r] = g.nz > 1 ? __dadd_rn(__dmul_rn(__dadd_rn(1.0, -zeta), lev[0]), __dmul_rn(zeta, lev[1]))
                        : lev[0];
    }
  }
  out = f.nt > 1 ? lerp_rn(val[0], val[1], tau) : val[0];
  return true;
}

}  // namespace pg
