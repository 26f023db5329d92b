// advect_plain.cuh -- the fused advection step for lon/lat/depth positions.
//
// One thread owns one particle for a whole chunk of steps (Eq. 1, Sect.
// 2.1.1): the particle state stays in registers, and so do the field values
// at the corners of the particle's current cell for the two bracketing
// snapshots.  A stage re-reads the field only when the particle has moved to
// another cell or another pair of snapshots, so the four RK4 stages of a step
// and consecutive steps inside one cell share one gather; when the pair of
// snapshots advances by one, the shared snapshot's corners are kept and only
// the new one is read.  The values used are the ones a fresh gather would
// return, so the arithmetic is that of the definition.
//
// Instantiated twice:
//   Real = double  (compiled with -fmad=false): the FP64 path, which carries
//     out the oracle's operations in the oracle's order, including the FP64
//     time interpolation of every stage and its cell and interval tie-breaks;
//   Real = float: the FP32 path, where stage times are FP32 offsets inside
//     the cached snapshot interval, cell and interval bounds are inclusive on
//     both sides (continuity makes the two choices at a shared node equal),
//     and no FP64 arithmetic runs per stage.
#pragma once

#include <type_traits>

#include "advect_common.cuh"

namespace pg {

// Locate p on the longitude axis, using and refreshing the cache.
// Returns false when the position is out of the domain.
template <typename Real, typename Store, int NF, bool D3, int GEO>
__device__ __forceinline__ bool locate_lon(const GridArgs &g, Sampler<Real, Store, NF, D3, GEO> &c,
                                           Real p, Real &xi) {
  Real q = p;
  const Real *x = axis<Real>(g, 0);
  if (is_per<GEO>(g)) {
    if (!isfinite(p)) return false;
    q = wrap_lon(p, axis_lo(g, 0, p));
  } else if (!(p >= axis_lo(g, 0, p) && p <= axis_hi(g, 0, p))) {
    return false;
  }
  if (!(c.ci >= 0 && in_cell<Real>(q, c.xlo, c.xhi, c.ci == g.nx - 2 && !is_per<GEO>(g)))) {
    c.dirty |= 1;
    if (is_per<GEO>(g) && q >= axis_hi(g, 0, p)) {
      c.ci = g.nx - 1;
      c.xlo = x[g.nx - 1];
      c.xhi = lon_end(g, p);
    } else {
      const int i = axis_search<Real>(g, 0, g.nx, q);
      c.ci = i;
      c.xlo = x[i]; c.xhi = x[i + 1];
    }
    c.rx = (Real)1 / (c.xhi - c.xlo);
  }
  if constexpr (sizeof(Real) == 8) xi = (q - c.xlo) / (c.xhi - c.xlo);
  else xi = (q - c.xlo) * c.rx;
  return true;
}

template <typename Real>
__device__ __forceinline__ bool locate_axis(const GridArgs &g, int a, int n, int &ci, Real &lo,
                                            Real &hi, Real &rinv, Real p, Real &xi, int &dirty) {
  const Real *x = axis<Real>(g, a);
  if (!(ci >= 0 && in_cell<Real>(p, lo, hi, ci == n - 2))) {
    if (!(p >= x[0] && p <= x[n - 1])) return false;
    const int i = axis_search<Real>(g, a, n, p);
    ci = i; lo = x[i]; hi = x[i + 1];
    dirty |= 1;
    rinv = (Real)1 / (hi - lo);
  }
  if constexpr (sizeof(Real) == 8) xi = (p - lo) / (hi - lo);
  else xi = (p - lo) * rinv;
  return true;
}

// FP32 slow path: locate p, known to lie outside the cached cell [lo, hi] of
// index ci on axis a (n nodes), and refresh the cell.  A move to a neighbour
// cell costs one node (the far node of the neighbour; the shared node is the
// old lo or hi); anything else searches the axis.  The cell found is the
// largest i <= n-2 with x[i] <= p, as a fresh search gives.  SELECT: both
// neighbours' far nodes are read (in bounds, usually L1 hits) and the move is
// selected without a branch -- measured faster in the 3-D kernel (fewer
// spills) and slower in the 2-D ones, which keep the branches; the cell
// found is the same either way.
template <bool SELECT>
__device__ __forceinline__ void relocate32(const GridArgs &g, int a, int n, float p, int &ci,
                                           float &lo, float &hi, float &rinv) {
  const float *x = axis<float>(g, a);
  if constexpr (SELECT) {
    const int cm = ci - 1 < 0 ? 0 : ci - 1;
    const int c2 = ci + 2 > n - 1 ? n - 1 : ci + 2;
    const float xm = x[cm], x2 = x[c2];
    const bool held = (ci >= 0) & (ci <= n - 2);
    const bool below = p < lo;
    const bool down = held & below & (ci >= 1) & (xm <= p);
    const bool up =
        held & !below & (ci + 1 <= n - 2) & ((p < x2) | ((ci + 1 == n - 2) & (p == x2)));
    int i = down ? ci - 1 : ci + 1;
    float nlo = down ? xm : hi, nhi = down ? lo : x2;
    if (!(down | up)) {
      i = axis_search<float>(g, a, n, p);
      nlo = x[i];
      nhi = x[i + 1];
    }
    ci = i;
    lo = nlo;
    hi = nhi;
    rinv = __frcp_rn(nhi - nlo);
    return;
  }
  int i = -1;
  float nlo = 0.f, nhi = 0.f;
  if (ci >= 0 && ci <= n - 2) {
    if (p < lo) {
      if (ci >= 1) {
        const float xm = x[ci - 1];
        if (xm <= p) { i = ci - 1; nlo = xm; nhi = lo; }
      }
    } else if (ci + 1 <= n - 2) {   // p > hi
      const float x2 = x[ci + 2];
      if (p < x2 || (ci + 1 == n - 2 && p == x2)) { i = ci + 1; nlo = hi; nhi = x2; }
    }
  }
  if (i < 0) {
    i = axis_search<float>(g, a, n, p);
    nlo = x[i];
    nhi = x[i + 1];
  }
  ci = i;
  lo = nlo;
  hi = nhi;
  rinv = __frcp_rn(nhi - nlo);   // correctly rounded, as 1.0f / (hi - lo)
}

// FP32: whether every stage time of a step of length h (offsets between 0
// and h from the step start) lies in the cached snapshot interval, so that
// the stages need not test it (a steady field always does).  A stage that
// leaves the interval finds it false and takes the slow path, which moves
// the interval; later stages of the step then take it too, at no cost in
// results.
template <typename Real, typename Store, int NF, bool D3, int GEO, class A>
__device__ __forceinline__ void step_in_interval(const A &a, const Sampler<Real, Store, NF, D3, GEO> &c,
                                                 Clock &ck, float h) {
  const float de = ck.d + h;
  ck.tin = (a.f.nt == 1) | ((c.s0 >= 0) & (fminf(ck.d, de) >= 0.f) & (fmaxf(ck.d, de) <= c.span));
}

// Velocity in position units per second at a stage (stage time = step start
// + off).  Returns 0 or a particle status (PG_OOB_*, PG_NAN); -1 for an
// internal failure already recorded in a.err.
template <bool EXT, typename Real, typename Store, int NF, bool D3, int GEO, class A>
__device__ __forceinline__ int velocity(const A &a, Sampler<Real, Store, NF, D3, GEO> &c,
                                        Clock &ck, Real off, Real lon, Real lat, Real dep,
                                        Real (&vel)[3]) {
  const GridArgs &g = a.g;
  if constexpr (sizeof(Real) == 4) {
    // FP32: one predicate tests the cached cell on every axis and whether the
    // whole step lies in the cached snapshot interval (ck.tin, set once per
    // step); only a miss runs the locate / interval / gather path, so the
    // common stage is one block without branches.  The longitude is tested
    // as it is: the cached cell lies in [x0, x0 + 360], so a position past
    // the zonal seam misses and the slow path reduces it.
    const float x0 = axis_lo(g, 0, lon);
    float q = lon;
    bool hit = (q >= c.xlo) & (q <= c.xhi) & (lat >= c.ylo) & (lat <= c.yhi);
    if constexpr (D3) hit = hit & (dep >= c.zlo) & (dep <= c.zhi);
    hit = hit & ck.tin;
    float xi, eta, zeta = 0.f;
    if (!hit) {
      // The stage velocities are not tested for NaN: a NaN velocity makes
      // the next stage position (or the step's result) NaN, which fails its
      // range test, and a failed test on a NaN position reports PG_NAN --
      // the status and the kept state of the definition's per-value test.
      // (Infinite velocities give infinite, not NaN, positions.)
      // each axis whose cached cell fails is located again (the Sampler
      // starts with empty cells on every axis, so all fail the first time)
      const int nan = (!(lon == lon) | !(lat == lat) | !(dep == dep)) ? 3 : 0;
      if (!((q >= c.xlo) & (q <= c.xhi))) {
        if (is_per<GEO>(g)) {
          if (!isfinite(lon)) return nan ? nan : 1;
          if (!(q >= x0 && q < x0 + 360.0f)) q = wrap_lon(lon, x0);
        } else if (!(lon >= x0 && lon <= axis_hi(g, 0, lon))) {
          return nan ? nan : 1;
        }
        c.dirty |= 1;
        if (is_per<GEO>(g) && q >= axis_hi(g, 0, q)) {   // the wrap cell
          c.ci = g.nx - 1;
          c.xlo = axis_hi(g, 0, q);
          c.xhi = lon_end(g, q);
          c.rx = __frcp_rn(c.xhi - c.xlo);
        } else {
          relocate32<D3>(g, 0, g.nx, q, c.ci, c.xlo, c.xhi, c.rx);
        }
      }
      if (!((lat >= c.ylo) & (lat <= c.yhi))) {
        if (!(lat >= axis_lo(g, 1, lat) && lat <= axis_hi(g, 1, lat))) return nan ? nan : 1;
        c.dirty |= 1;
        relocate32<D3>(g, 1, g.ny, lat, c.cj, c.ylo, c.yhi, c.ry);
      }
      if constexpr (D3) {
        if (!((dep >= c.zlo) & (dep <= c.zhi))) {
          if (!(dep >= axis_lo(g, 2, dep) && dep <= axis_hi(g, 2, dep))) return nan ? nan : 2;
          c.dirty |= 1;
          relocate32<D3>(g, 2, g.nz, dep, c.ck, c.zlo, c.zhi, c.rz);
        }
      } else {
        c.ck = 0;
      }
      if (refresh32(a, c, ck, off)) return -1;
    }
    xi = (q - c.xlo) * c.rx;
    eta = (lat - c.ylo) * c.ry;
    if constexpr (D3) zeta = (dep - c.zlo) * c.rz;
    if constexpr (EXT) {
      if (a.f.nearest) nearest32(c, xi, eta, zeta, tau32(a, c, ck, off), vel);
      else interp32<Store, NF, D3, GEO, false>(c, xi, eta, zeta, tau32(a, c, ck, off), vel);
    } else {
      const int r = interp32<Store, NF, D3, GEO, false>(c, xi, eta, zeta, tau32(a, c, ck, off), vel);
      if (r) return r;
    }
    if (is_sph<GEO>(g)) {
      vel[0] = lon_rate(vel[0], lat, a.k);
      vel[1] = lat_rate(vel[1], a.k);
    }
    return 0;
  }
  Real xi, eta, zeta = (Real)0;
  if (!locate_lon(g, c, lon, xi)) return 1;
  if (!locate_axis<Real>(g, 1, g.ny, c.cj, c.ylo, c.yhi, c.ry, lat, eta, c.dirty)) return 1;
  if constexpr (D3) {
    if (!locate_axis<Real>(g, 2, g.nz, c.ck, c.zlo, c.zhi, c.rz, dep, zeta, c.dirty)) return 2;
  } else {
    c.ck = 0;
  }
  const int r = sample_fields(a, c, ck, off, xi, eta, zeta, vel);
  if (r) return r;
  if (is_sph<GEO>(g)) {
    vel[0] = lon_rate(vel[0], lat, a.k);
    vel[1] = lat_rate(vel[1], a.k);
  }
  return 0;
}

// Parameters of the worked example's behaviours per Real.
__device__ __forceinline__ double dwell_of(const KernArgs &k, double) { return k.dwell; }
__device__ __forceinline__ float dwell_of(const KernArgs &k, float) { return k.dwell_f; }

template <bool EXT, typename Real, typename Store, int NF, bool D3, int GEO, class A>
__device__ __forceinline__ int finish_step(const A &a, Real &lon, Real &lat, Real &dep, Real nlon,
                                           Real nlat, Real ndep, Real hr, double h64,
                                           double &age, const uint64_t *idp, uint32_t stp);

// One step of Eq. 1.  Returns 0 and updates (lon, lat, dep) on success.
// RK4 stages run in a loop: stage s samples at (X + k_{s-1} c_s h, t + c_s h)
// with c = (0, 1/2, 1/2, 1) and accumulates ((k1 + 2 k2) + 2 k3) + k4.
// With the worked example's behaviours (EXT, and always in FP64): settle
// after sinking; after the step is applied, age += |h| (the step's exact FP64
// length h64) and STATUS_DELETED is returned, state updated, once the age
// reaches the maximum.
template <bool EXT, typename Real, typename Store, int NF, bool D3, int GEO, class A>
__device__ __forceinline__ int step_one(const A &a, Sampler<Real, Store, NF, D3, GEO> &c,
                                        Clock &ck, Real &lon, Real &lat, Real &dep, Real hr,
                                        double h64, double &age, const uint64_t *idp,
                                        uint32_t stp) {
  constexpr bool X = EXT || sizeof(Real) == 8;
  Real kc[3] = {(Real)0, (Real)0, (Real)0};
  Real acc[3];
  const Real half = (Real)0.5 * hr;
  const int nst = a.k.scheme == 0 ? 1 : 4;
  int r;
  if constexpr (sizeof(Real) == 4) {
    // FP32: the same sums without branches on the stage: offsets c_s h with
    // c = (0, 1/2, 1/2, 1), weights (1, 2, 2, 1); 2 k and c_s h are exact
    acc[0] = 0.f; acc[1] = 0.f; acc[2] = 0.f;
    step_in_interval(a, c, ck, hr);
#pragma unroll 1
    for (int s = 0; s < nst; ++s) {
      const float off = (s == 0 ? 0.f : (s == 3 ? 1.f : 0.5f)) * hr;
      const float px = fmaf(kc[0], off, lon), py = fmaf(kc[1], off, lat);
      const float pz = fmaf(kc[2], off, dep);
      if ((r = velocity<EXT>(a, c, ck, off, px, py, pz, kc))) return r;
      const float wg = (s == 1 || s == 2) ? 2.f : 1.f;
      acc[0] = fmaf(wg, kc[0], acc[0]);
      acc[1] = fmaf(wg, kc[1], acc[1]);
      acc[2] = fmaf(wg, kc[2], acc[2]);
    }
  } else
#pragma unroll 1
  for (int s = 0; s < nst; ++s) {
    const Real off = s == 0 ? (Real)0 : (s == 3 ? hr : half);
    Real px = lon, py = lat, pz = dep;
    if (s > 0) {
      px = lon + kc[0] * off;
      py = lat + kc[1] * off;
      pz = dep + kc[2] * off;
    }
    if ((r = velocity<EXT>(a, c, ck, off, px, py, pz, kc))) return r;
    if (s == 0) {
      acc[0] = kc[0]; acc[1] = kc[1]; acc[2] = kc[2];
    } else if (s == 3) {
      acc[0] = acc[0] + kc[0]; acc[1] = acc[1] + kc[1]; acc[2] = acc[2] + kc[2];
    } else {
      acc[0] = acc[0] + (Real)2 * kc[0];
      acc[1] = acc[1] + (Real)2 * kc[1];
      acc[2] = acc[2] + (Real)2 * kc[2];
    }
  }
  Real nlon, nlat, ndep;
  if constexpr (sizeof(Real) == 4) {
    // FP32: (k1 + 2 k2 + 2 k3 + k4) h / 6 with h / 6 formed once (no division)
    const float w = nst == 1 ? hr : hr * (1.0f / 6.0f);
    nlon = fmaf(acc[0], w, lon);
    nlat = fmaf(acc[1], w, lat);
    ndep = fmaf(acc[2], w, dep);
  } else if (nst == 1) {
    nlon = lon + acc[0] * hr;
    nlat = lat + acc[1] * hr;
    ndep = dep + acc[2] * hr;
  } else {
    nlon = lon + acc[0] / (Real)6 * hr;
    nlat = lat + acc[1] / (Real)6 * hr;
    ndep = dep + acc[2] / (Real)6 * hr;
  }
  return finish_step<EXT, Real, Store, NF, D3, GEO>(a, lon, lat, dep, nlon, nlat, ndep, hr, h64,
                                                    age, idp, stp);
}

// The part of a step after advection, from the advected position (nlon,
// nlat, ndep): behaviours (Brownian, sinking; settle), the zonal wrap, the
// domain test; on success the new state and the age.  Returns 0, a status
// (state untouched), or STATUS_DELETED (state updated).
template <bool EXT, typename Real, typename Store, int NF, bool D3, int GEO, class A>
__device__ __forceinline__ int finish_step(const A &a, Real &lon, Real &lat, Real &dep, Real nlon,
                                           Real nlat, Real ndep, Real hr, double h64,
                                           double &age, const uint64_t *idp, uint32_t stp) {
  constexpr bool X = EXT || sizeof(Real) == 8;
  int r;
  if (a.k.beh & 1u) {
    Real n1, n2;
    normal_pair(a.k.seed, *idp, stp, n1, n2);
    const Real sigma = pg_sqrt((Real)2 * kh_of(a.k, hr) * pg_fabs(hr));
    Real dx = sigma * n1, dy = sigma * n2;
    if (is_sph<GEO>(a.g)) {
      dx = lon_rate(dx, nlat, a.k);
      dy = lat_rate(dy, a.k);
    }
    nlon = nlon + dx;
    nlat = nlat + dy;
  }
  if (a.k.beh & 2u) ndep = ndep + w_of(a.k, hr) * hr;
  bool dwelling = false;   // settle: the step starts at the dwelling depth
  if constexpr (X) {
    if (a.k.beh & BEH_SETTLE) {
      const Real zd = dwell_of(a.k, hr);
      if (dep == zd) {
        dwelling = true;
        ndep = zd;
      } else {
        Real moved = ndep + w_of(a.k, hr) * hr;
        if ((dep - zd) * (moved - zd) <= (Real)0) moved = zd;
        ndep = moved;
      }
    }
  }
  if (is_per<GEO>(a.g)) nlon = wrap_lon(nlon, axis_lo(a.g, 0, nlon));
  if ((r = out_of_domain<Real, GEO>(a.g, nlon, nlat, ndep, D3))) {
    // FP32: a NaN result comes from a NaN stage velocity (see velocity)
    if constexpr (sizeof(Real) == 4) {
      if (!(nlon == nlon) | !(nlat == nlat) | !(ndep == ndep)) return 3;
    }
    return r;
  }
  lon = nlon; lat = nlat; dep = ndep;
  if constexpr (X) {
    if (a.k.beh & BEH_AGE) {
      if (!(a.k.beh & BEH_SETTLE) || dwelling) age = age + fabs(h64);
      if (age >= a.k.max_age) return STATUS_DELETED;
    }
  }
  return 0;
}

// ------------------------------------------------------------------ RKF45
// The Fehlberg 4(5) pair (Sect. 2.1.1 names Runge-Kutta-Fehlberg): stage
// times, stage weights, fourth- and fifth-order weights, in FP64 and FP32.
// Fourth- and fifth-order weights (read in unrolled code).
__device__ constexpr double kRkfB4[6] = {25.0 / 216.0, 0.0, 1408.0 / 2565.0, 2197.0 / 4104.0,
                                         -1.0 / 5.0, 0.0};
__device__ constexpr double kRkfB5[6] = {16.0 / 135.0, 0.0, 6656.0 / 12825.0,
                                         28561.0 / 56430.0, -9.0 / 50.0, 2.0 / 55.0};
// Stage times and stage weights (read with the stage as a runtime index).
__device__ constexpr double kRkfC64[6] = {0.0, 1.0 / 4.0, 3.0 / 8.0, 12.0 / 13.0, 1.0, 1.0 / 2.0};
__device__ constexpr double kRkfA64[6][5] = {
    {0, 0, 0, 0, 0},
    {1.0 / 4.0, 0, 0, 0, 0},
    {3.0 / 32.0, 9.0 / 32.0, 0, 0, 0},
    {1932.0 / 2197.0, -7200.0 / 2197.0, 7296.0 / 2197.0, 0, 0},
    {439.0 / 216.0, -8.0, 3680.0 / 513.0, -845.0 / 4104.0, 0},
    {-8.0 / 27.0, 2.0, -3544.0 / 2565.0, 1859.0 / 4104.0, -11.0 / 40.0}};
__device__ constexpr float kRkfC32[6] = {0.0f, (float)(1.0 / 4.0), (float)(3.0 / 8.0),
                                         (float)(12.0 / 13.0), 1.0f, 0.5f};
__device__ constexpr float kRkfA32[6][5] = {
    {0, 0, 0, 0, 0},
    {(float)(1.0 / 4.0), 0, 0, 0, 0},
    {(float)(3.0 / 32.0), (float)(9.0 / 32.0), 0, 0, 0},
    {(float)(1932.0 / 2197.0), (float)(-7200.0 / 2197.0), (float)(7296.0 / 2197.0), 0, 0},
    {(float)(439.0 / 216.0), -8.0f, (float)(3680.0 / 513.0), (float)(-845.0 / 4104.0), 0},
    {(float)(-8.0 / 27.0), 2.0f, (float)(-3544.0 / 2565.0), (float)(1859.0 / 4104.0),
     (float)(-11.0 / 40.0)}};
__device__ __forceinline__ double rkf_c(int i, double) { return kRkfC64[i]; }
__device__ __forceinline__ float rkf_c(int i, float) { return kRkfC32[i]; }
__device__ __forceinline__ double rkf_a(int i, int j, double) { return kRkfA64[i][j]; }
__device__ __forceinline__ float rkf_a(int i, int j, float) { return kRkfA32[i][j]; }

// One trial of length h from (lon, lat, dep) at the clock's step start: the
// fourth-order position x4 and the error estimate in metres (the largest
// over the axes of |X5 - X4|, degrees turned into metres at the latitude of
// X4 on a sphere).  The six stages run in a loop that is not unrolled (one
// copy of the velocity code); each stage's slopes go to its own registers,
// and the stage position adds h a_ij k_j over the earlier stages j in order
// (later ones have zero weight and zero slopes, which add exactly zero).
// Returns 0, a particle status, or -1 (internal failure).
template <bool EXT, typename Real, typename Store, int NF, bool D3, int GEO, class A>
__device__ __forceinline__ int rkf45_trial(const A &a, Sampler<Real, Store, NF, D3, GEO> &c,
                                           Clock &ck, Real lon, Real lat, Real dep, Real h,
                                           Real (&x4)[3], Real &err) {
  Real kx[6], ky[6], kz[6];
#pragma unroll
  for (int j = 0; j < 6; ++j) { kx[j] = (Real)0; ky[j] = (Real)0; kz[j] = (Real)0; }
  int r;
#pragma unroll 1
  for (int i = 0; i < 6; ++i) {
    Real px = lon, py = lat, pz = dep;
#pragma unroll
    for (int j = 0; j < 5; ++j) {
      const Real ha = h * rkf_a(i, j, h);
      px = px + ha * kx[j];
      py = py + ha * ky[j];
      pz = pz + ha * kz[j];
    }
    Real kn[3];
    if ((r = velocity<EXT>(a, c, ck, rkf_c(i, h) * h, px, py, pz, kn))) return r;
#pragma unroll
    for (int j = 0; j < 6; ++j) {
      if (i == j) { kx[j] = kn[0]; ky[j] = kn[1]; kz[j] = kn[2]; }
    }
  }
  Real d4[3] = {(Real)0, (Real)0, (Real)0}, d5[3] = {(Real)0, (Real)0, (Real)0};
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    d4[0] = d4[0] + (Real)kRkfB4[i] * kx[i];
    d4[1] = d4[1] + (Real)kRkfB4[i] * ky[i];
    d4[2] = d4[2] + (Real)kRkfB4[i] * kz[i];
    d5[0] = d5[0] + (Real)kRkfB5[i] * kx[i];
    d5[1] = d5[1] + (Real)kRkfB5[i] * ky[i];
    d5[2] = d5[2] + (Real)kRkfB5[i] * kz[i];
  }
  x4[0] = lon + h * d4[0];
  x4[1] = lat + h * d4[1];
  x4[2] = dep + h * d4[2];
  Real ex = pg_fabs(h * (d5[0] - d4[0])), ey = pg_fabs(h * (d5[1] - d4[1]));
  const Real ez = pg_fabs(h * (d5[2] - d4[2]));
  if (is_sph<GEO>(a.g)) {
    ex = ex * (Real)a.k.deg_m * cos_deg(x4[1]);
    ey = ey * (Real)a.k.deg_m;
  }
  const Real e = ex > ey ? ex : ey;
  err = e > ez ? e : ez;
  return 0;
}

// RKF45 steps of one particle while its time lies before t_stop and t_end:
// trials rejected above the tolerance halve the particle's step length, an
// accepted full-length step with a tenth of the tolerance doubles it, and
// steps are shortened to land on t_clip (the next output time) and t_end.
// Returns the steps taken; writes the state, status and step length back
// through the references.
template <bool EXT, typename Real, typename Store, int NF, bool D3, int GEO, class A>
__device__ __forceinline__ unsigned long long rkf45_steps(
    const A &a, Sampler<Real, Store, NF, D3, GEO> &c, Real &lon, Real &lat, Real &dep, double &t,
    uint32_t &stp, double &hp, double &age, uint8_t &st, const uint64_t *idp) {
  const double sgn = a.dt > 0.0 ? 1.0 : -1.0;
  if (!(sgn * hp > 0.0)) hp = a.dt;
  const double target = sgn * (a.t_clip - a.t_end) < 0.0 ? a.t_clip : a.t_end;
  unsigned long long done = 0;
  Clock ck;
  ck.dt = 0.0; ck.k = 0;
  while (sgn * (a.t_stop - t) > 0.0 && sgn * (a.t_end - t) > 0.0) {
    double h = hp;
    bool clipped = false;
    if (sgn * (target - t) < sgn * h) { h = target - t; clipped = true; }
    ck.t = t;
    if constexpr (sizeof(Real) == 4) {
      ck.d = c.s0 >= 0 ? (float)(t - c.ta) : 0.f;
      step_in_interval(a, c, ck, (float)h);
    }
    Real x4[3], err;
    int r = rkf45_trial<EXT>(a, c, ck, lon, lat, dep, (Real)h, x4, err);
    if (r > 0) { st = (uint8_t)r; break; }
    if (r < 0) break;
    if ((double)err > a.k.rk_tol && fabs(h) > a.k.rk_hmin) {
      hp = sgn * fmax(fabs(h) / 2.0, a.k.rk_hmin);
      continue;
    }
    r = finish_step<EXT, Real, Store, NF, D3, GEO>(a, lon, lat, dep, x4[0], x4[1], x4[2],
                                                  (Real)h, h, age, idp, stp);
    if (r > 0 && r != STATUS_DELETED) { st = (uint8_t)r; break; }
    t = t + h;
    ++stp;
    ++done;
    if (!clipped && (double)err < a.k.rk_tol / 10.0) hp = sgn * fmin(2.0 * fabs(hp), a.k.rk_hmax);
    if (r == STATUS_DELETED) { st = (uint8_t)r; break; }
  }
  return done;
}

// Scalar fields sampled at a particle's state into its variables (the
// sample behaviour).  Sampling after every step and sampling once at the end
// of a chunk give the same variables: each sample overwrites the last, and
// the state at the end of the chunk is the state after its last step.
template <typename Store, class A>
__device__ __forceinline__ void sample_variables(const A &a, int64_t p, double lon, double lat,
                                                 double dep, double t) {
  using TS = typename std::conditional<std::is_same<Store, double>::value, double, float>::type;
  for (int q = 0; q < a.f.ntr; ++q) {
    double v;
    if (tracer_value<TS>(a.g, a.f, q, lon, lat, dep, t, v, a.err)) a.p.var[q * a.p.vstride + p] = v;
  }
}

// The chunk kernel: each thread advances one particle while its time is
// before t_stop and t_end (in the direction of dt), shortening only the step
// that lands on t_end.  Returns the number of steps taken.
template <bool EXT, typename Real, typename Store, int NF, bool D3, int GEO, class A>
__device__ __forceinline__ unsigned long long advance_particle(const A &a, int64_t p) {
  constexpr bool X = EXT || sizeof(Real) == 8;
  unsigned long long done = 0;
  {
    double age = 0.0;
    if constexpr (X) {
      if (a.k.beh & BEH_AGE) age = a.p.age[p];
    }
    Real *PX = reinterpret_cast<Real *>(a.p.x);
    Real *PY = reinterpret_cast<Real *>(a.p.y);
    Real *PZ = reinterpret_cast<Real *>(a.p.z);
    Real lon = PX[p], lat = PY[p], dep = PZ[p];
    double t = a.p.time[p];
    uint32_t stp = a.p.step[p];
    const uint64_t *idp = a.p.id + p;   // read by the Brownian step only
    uint8_t st = 0;
    Sampler<Real, Store, NF, D3, GEO> c;
    c.reset();
    const double sgn = a.dt > 0.0 ? 1.0 : -1.0;
    Clock ck;
    ck.dt = a.dt; ck.k = 0; ck.d = 0.f;
    bool adaptive = false;
    if constexpr (X) adaptive = a.k.scheme == 2;
    if (adaptive) {
      if constexpr (X) {
        double hp = a.p.hstep[p];
        done = rkf45_steps<EXT>(a, c, lon, lat, dep, t, stp, hp, age, st, idp);
        a.p.hstep[p] = hp;
      }
    } else if constexpr (sizeof(Real) == 8) {
      // FP64: the definition's loop, time accumulated step by step.
      while (sgn * (a.t_stop - t) > 0.0 && sgn * (a.t_end - t) > 0.0) {
        double h = a.dt;
        if (sgn * (a.t_end - t) < sgn * h) h = a.t_end - t;
        ck.t = t;
        const int r = step_one<EXT>(a, c, ck, lon, lat, dep, (Real)h, h, age, idp, stp);
        if (r == STATUS_DELETED) {      // taken, then deleted by the age behaviour
          t = t + h;
          ++stp;
          ++done;
          st = (uint8_t)r;
          break;
        }
        if (r > 0) { st = (uint8_t)r; break; }
        if (r < 0) break;
        t = t + h;
        ++stp;
        ++done;
      }
    } else {
      // FP32: the step count of this chunk is fixed up front; step k starts
      // at t + k dt (exact for times and steps in whole seconds), and only
      // a step that lands on t_end is shortened.
      const double tl = sgn > 0.0 ? fmin(a.t_stop, a.t_end) : fmax(a.t_stop, a.t_end);
      int n = 0;
      if (sgn * (tl - t) > 0.0) n = (int)ceil((tl - t) / a.dt);
      double hlast = a.dt;
      if (n > 0 && sgn * (a.t_end - (t + (double)(n - 1) * a.dt)) < sgn * a.dt)
        hlast = a.t_end - (t + (double)(n - 1) * a.dt);
      const float hf = (float)a.dt, hlf = (float)hlast;
      ck.t = t;
      int k = 0;
      for (; k < n; ++k) {
        ck.k = k;
        const float h = (k == n - 1) ? hlf : hf;
        const int r = step_one<EXT>(a, c, ck, lon, lat, dep, (Real)h,
                                    (k == n - 1) ? hlast : a.dt, age, idp, stp);
        if (r > 0) {
          if (X && r == STATUS_DELETED) {   // taken, then deleted by the age behaviour
            ++stp;
            ck.d += h;
            ++k;
          }
          st = (uint8_t)r;
          break;
        }
        if (r < 0) break;
        ++stp;
        ck.d += h;
      }
      done = (unsigned long long)k;
      if (k == n && n > 0) t = (hlast != a.dt) ? a.t_end : t + (double)n * a.dt;
      else t = t + (double)k * a.dt;
    }
    PX[p] = lon; PY[p] = lat; PZ[p] = dep;
    a.p.time[p] = t;
    a.p.step[p] = stp;
    a.p.status[p] = st;
    if constexpr (X) {
      if (a.k.beh & BEH_AGE) a.p.age[p] = age;
      if ((a.k.beh & BEH_SAMPLE) && done > 0)
        sample_variables<Store>(a, p, (double)lon, (double)lat, (double)dep, t);
    }
  }
  return done;
}

// One atomic per warp for the particle-step counter.
__device__ __forceinline__ void count_steps(unsigned long long done, unsigned long long *counter) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) done += __shfl_down_sync(0xffffffffu, done, o);
  if ((threadIdx.x & 31) == 0 && done) atomicAdd(counter, done);
}

// FP32 3-D: at most 128 registers (two 256-thread blocks per SM); measured
// faster than the unbounded allocation despite a few spilled words, as more
// resident warps hide the gather and dependency latencies.  FP32 2-D: at most
// 72 registers, seven 128-thread blocks (28 warps) per SM (1.2 % faster than six
// on the 1/12-degree workload, a few spilled words); with the worked
// example's behaviours, six.
//
// EXT = true: the FP32 kernel with the worked example's behaviours (settle,
// age, sampled variables) and nearest-neighbour interpolation; the FP64
// kernel always has them.
template <typename Real, typename Store, int NF, bool D3, int GEO, bool EXT = false>
__global__ void __launch_bounds__(sizeof(Real) == 4 && !D3 ? 128 : 256,
                                  sizeof(Real) == 4 ? (D3 ? 2 : (EXT ? 6 : 7)) : 1)
    advect_plain_kernel(StepArgs a) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  unsigned long long done = 0;
  if (p < a.p.n && a.p.status[p] == 0) done = advance_particle<EXT, Real, Store, NF, D3, GEO>(a, p);
  count_steps(done, a.steps_done);
}

// Batched form: a persistent kernel walks a device work list of tiles
// (release, first particle); each CTA takes the next tile with one atomic,
// so releases of very different cost (dt from 10 min to 2 h) balance across
// the SMs.  Each release brings its own particle arrays, kernel, dt and end
// time (table `rel`); the field is shared.
struct BatchRelease {
  PartArgs p;
  KernArgs k;
  double dt, t_end;
};

struct BatchArgs {
  GridArgs g;
  FieldArgs f;
  const BatchRelease *rel;
  const int2 *tiles;      // (release, first particle), heaviest first
  int ntiles;
  int *next_tile;         // work-list cursor, zeroed before every launch
  double t_stop;
  unsigned long long *steps_done;
  int *err;
};

// The step's arguments as the batch kernel sees them: the grid and the field
// refer to the kernel's parameters (constant bank), the release's kernel and
// particle arrays to the copy the tile's first thread made in shared memory.
struct BatchStep {
  const GridArgs &g;
  const FieldArgs &f;
  const KernArgs &k;
  const PartArgs &p;
  double dt, t_stop, t_end;
  unsigned long long *steps_done;
  int *err;
};

template <typename Store, int NF, bool D3, int GEO>
__global__ void __launch_bounds__(256, 2) advect_batch_kernel(const __grid_constant__ BatchArgs b) {
  __shared__ int tile;
  __shared__ KernArgs sk;
  __shared__ PartArgs sp;
  __shared__ double sdt, st_end;
  unsigned long long done = 0;
  for (;;) {
    if (threadIdx.x == 0) {
      tile = atomicAdd(b.next_tile, 1);
      if (tile < b.ntiles) {
        const BatchRelease *R = b.rel + b.tiles[tile].x;
        sk = R->k;
        sp = R->p;
        sdt = R->dt;
        st_end = R->t_end;
      }
    }
    __syncthreads();
    const int t = tile;
    if (t >= b.ntiles) break;
    const BatchStep v{b.g, b.f, sk, sp, sdt, b.t_stop, st_end, b.steps_done, b.err};
    const int64_t p = (int64_t)b.tiles[t].y + threadIdx.x;
    if (p < sp.n && sp.status[p] == 0) done += advance_particle<false, float, Store, NF, D3, GEO>(v, p);
    __syncthreads();
  }
  count_steps(done, b.steps_done);
}

}  // namespace pg
