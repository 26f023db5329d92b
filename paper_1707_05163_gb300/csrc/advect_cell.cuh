// advect_cell.cuh -- the fused advection step for positions stored as an
// integer cell index plus an FP32 offset inside the cell (uniform axes).
//
// On uniformly spaced axes the index coordinate X = (x - x0) / dx is an
// affine map of the position, so RK4 (Sect. 2.1.1) gives the same path in
// index units with velocities divided by the spacing (RK4 commutes with
// affine maps).  Storing the integer part separately keeps an FP32 offset
// resolution of 2^-24 cell anywhere on the globe (an FP32 longitude near 360
// degrees resolves only 3e-5 degrees), and the cell of every stage follows
// from the base cell and the offset without any search.  Field storage may be
// FP32, FP16 or BF16 (values = code * per-snapshot scale).
#pragma once

#include "advect_common.cuh"

namespace pg {

struct CellState {
  int i, j, k;
  float x, y, z;
};

// Move an offset into [0, 1), carrying whole cells into the index.  Periodic
// axes wrap the index into [0, n); others must stay inside [0, n-1], the last
// node itself being offset 1 of cell n-2.  Returns false when outside.
__device__ __forceinline__ bool norm_axis(int &i, float &f, int n, bool periodic) {
  if (!(f >= 0.f && f < 1.f)) {
    if (!(fabsf(f) < 1.0e6f)) return false;   // also NaN
    const float fl = floorf(f);
    i += (int)fl;
    f -= fl;
    if (f >= 1.f) { f = 0.f; i += 1; }
  }
  if (periodic) {
    if (i < 0) i += n * ((-i + n - 1) / n);
    else if (i >= n) i -= n * (i / n);
    return true;
  }
  if (i >= 0 && i <= n - 2) return true;
  if (i == n - 1 && f == 0.f) { i = n - 2; f = 1.f; return true; }
  return false;
}

// Velocity in cells per second at the stage position base + kc * off.
template <typename Store, int NF, bool D3, int GEO>
__device__ __forceinline__ int velocity_cell(const StepArgs &a, Sampler<float, Store, NF, D3, GEO> &c,
                                             Clock &ck, float off, const CellState &b,
                                             const float (&kc)[3], float (&vel)[3]) {
  const GridArgs &g = a.g;
  int i = b.i, j = b.j, k = b.k;
  float x = b.x + kc[0] * off, y = b.y + kc[1] * off, z = D3 ? b.z + kc[2] * off : 0.f;
  // No NaN test on the stage velocity: a NaN velocity makes the next stage
  // offset (or the step's result) NaN, which fails normalisation, and a
  // failure on a NaN offset reports PG_NAN, with the state kept.
  const int nan = (!(x == x) | !(y == y) | !(z == z)) ? 3 : 0;
  if (!norm_axis(i, x, g.nx, is_per<GEO>(g))) return nan ? nan : 1;
  if (!norm_axis(j, y, g.ny, false)) return nan ? nan : 1;
  if constexpr (D3) {
    if (!norm_axis(k, z, g.nz, false)) return nan ? nan : 2;
  }
  if (i != c.ci || j != c.cj || (D3 && k != c.ck)) {
    c.ci = i;
    c.cj = j;
    c.ck = D3 ? k : 0;
    c.dirty |= 1;
  }
  if (refresh32(a, c, ck, off)) return -1;
  interp32<Store, NF, D3, GEO, false>(c, x, y, z, tau32(a, c, ck, off), vel);
  if (is_sph<GEO>(g)) {
    const float lat = g.x0f[1] + ((float)j + y) * g.df[1];
    vel[0] = __fdividef(vel[0] * g.inv_m[0], cos_deg(lat));
  } else {
    vel[0] = vel[0] * g.inv_m[0];
  }
  vel[1] = vel[1] * g.inv_m[1];
  vel[2] = vel[2] * g.inv_m[2];
  return 0;
}

// One step of Eq. 1 in cell units; the state is replaced only on success.
template <typename Store, int NF, bool D3, int GEO>
__device__ __forceinline__ int step_cell(const StepArgs &a, Sampler<float, Store, NF, D3, GEO> &c,
                                         Clock &ck, CellState &s, float h, const uint64_t *idp,
                                         uint32_t stp) {
  const GridArgs &g = a.g;
  float kc[3] = {0.f, 0.f, 0.f};
  float acc[3];
  const float half = 0.5f * h;
  const int nst = a.k.scheme == 0 ? 1 : 4;
  int r;
  acc[0] = 0.f; acc[1] = 0.f; acc[2] = 0.f;
#pragma unroll 1
  for (int q = 0; q < nst; ++q) {
    const float off = (q == 0 ? 0.f : (q == 3 ? 1.f : 0.5f)) * h;
    if ((r = velocity_cell(a, c, ck, off, s, kc, kc))) return r;
    const float wg = (q == 1 || q == 2) ? 2.f : 1.f;
    acc[0] = fmaf(wg, kc[0], acc[0]);
    acc[1] = fmaf(wg, kc[1], acc[1]);
    acc[2] = fmaf(wg, kc[2], acc[2]);
  }
  const float w = nst == 1 ? h : h * (1.0f / 6.0f);
  CellState n = s;
  n.x = s.x + acc[0] * w;
  n.y = s.y + acc[1] * w;
  n.z = D3 ? s.z + acc[2] * w : 0.f;
  if (a.k.beh & 1u) {
    float n1, n2;
    normal_pair(a.k.seed, *idp, stp, n1, n2);
    const float sigma = sqrtf(2.f * a.k.kh_f * fabsf(h));
    float dx = sigma * n1 * g.inv_m[0];
    if (is_sph<GEO>(g)) dx = __fdividef(dx, cos_deg(g.x0f[1] + ((float)n.j + n.y) * g.df[1]));
    n.x += dx;
    n.y += sigma * n2 * g.inv_m[1];
  }
  if (D3 && (a.k.beh & 2u)) n.z += a.k.w_sink_f * h * g.inv_m[2];
  // a NaN result comes from a NaN stage velocity (see velocity_cell)
  if (!(n.x == n.x) | !(n.y == n.y) | !(n.z == n.z)) return 3;
  if (!norm_axis(n.i, n.x, g.nx, is_per<GEO>(g))) return 1;
  if (!norm_axis(n.j, n.y, g.ny, false)) return 1;
  if constexpr (D3) {
    if (!norm_axis(n.k, n.z, g.nz, false)) return 2;
  }
  s = n;
  return 0;
}

template <typename Store, int NF, bool D3, int GEO>
// 3-D: at most 128 registers (two 256-thread blocks per SM).  2-D, with a
// third of the corner values: at most 85 registers, six 128-thread blocks
// (24 warps) per SM, measured faster than five or four.
__global__ void __launch_bounds__(D3 ? 256 : 128, D3 ? 2 : 6) advect_cell_kernel(StepArgs a) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  unsigned long long done = 0;
  if (p < a.p.n && a.p.status[p] == 0) {
    CellState s;
    s.i = a.p.ci[p]; s.j = a.p.cj[p]; s.x = a.p.fx[p]; s.y = a.p.fy[p];
    if (D3) { s.k = a.p.ck[p]; s.z = a.p.fz[p]; } else { s.k = 0; s.z = 0.f; }
    double t = a.p.time[p];
    uint32_t stp = a.p.step[p];
    const uint64_t *idp = a.p.id + p;   // read by the Brownian step only
    uint8_t st = 0;
    Sampler<float, Store, NF, D3, GEO> c;
    c.reset();
    const double sgn = a.dt > 0.0 ? 1.0 : -1.0;
    // the step count of this chunk is fixed up front; step k starts at
    // t + k dt, and only a step that lands on t_end is shortened
    const double tl = sgn > 0.0 ? fmin(a.t_stop, a.t_end) : fmax(a.t_stop, a.t_end);
    int n = 0;
    if (sgn * (tl - t) > 0.0) n = (int)ceil((tl - t) / a.dt);
    double hlast = a.dt;
    if (n > 0 && sgn * (a.t_end - (t + (double)(n - 1) * a.dt)) < sgn * a.dt)
      hlast = a.t_end - (t + (double)(n - 1) * a.dt);
    const float hf = (float)a.dt, hlf = (float)hlast;
    Clock ck;
    ck.t = t; ck.dt = a.dt; ck.k = 0; ck.d = 0.f;
    int k = 0;
    for (; k < n; ++k) {
      ck.k = k;
      const float h = (k == n - 1) ? hlf : hf;
      const int r = step_cell(a, c, ck, s, h, idp, stp);
      if (r > 0) { st = (uint8_t)r; break; }
      if (r < 0) break;
      ++stp;
      ck.d += h;
    }
    done = (unsigned long long)k;
    if (k == n && n > 0) t = (hlast != a.dt) ? a.t_end : t + (double)n * a.dt;
    else t = t + (double)k * a.dt;
    a.p.ci[p] = s.i; a.p.cj[p] = s.j; a.p.fx[p] = s.x; a.p.fy[p] = s.y;
    if (D3) { a.p.ck[p] = s.k; a.p.fz[p] = s.z; }
    a.p.time[p] = t;
    a.p.step[p] = stp;
    a.p.status[p] = st;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) done += __shfl_down_sync(0xffffffffu, done, o);
  if ((threadIdx.x & 31) == 0 && done) atomicAdd(a.steps_done, done);
}

}  // namespace pg
