// capi.cu -- the C ABI: field sets, kernels, particle sets and the time loop.
//
// The objects follow the FieldSet / ParticleSet / Kernel / execute statement
// of the problem in Lange & van Sebille, "Parcels v0.9" (Sect. 2.1, 2.2, 2.4
// and 3).  The time loop advances particles in chunks of steps (one kernel
// launch each); chunks end at output times, at re-sort times and, for
// streamed fields, at snapshot times, so that the snapshots a chunk needs are
// resident before it starts while the next one uploads on a side stream.
#include <cstdarg>
#include <cstdio>
#include <cstring>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <limits>

#include "pg_host.h"

namespace pg {

static thread_local std::string g_err;
static int64_t g_alloc_limit = -1;      // test hook: fail allocations beyond this
static int64_t g_alloc_bytes = 0;
static std::atomic<long long> g_launches{0};

void note_launches(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

void set_error(const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
}
void clear_error() { g_err.clear(); }

cudaError_t dev_alloc(void **p, size_t bytes) {
  *p = nullptr;
  if (bytes == 0) bytes = 16;
  if (g_alloc_limit >= 0 && g_alloc_bytes + (int64_t)bytes > g_alloc_limit)
    return cudaErrorMemoryAllocation;
  cudaError_t e = cudaMalloc(p, bytes);
  if (e == cudaSuccess) g_alloc_bytes += (int64_t)bytes;
  return e;
}
void dev_free(void *p) {
  if (p) cudaFree(p);
}

cudaError_t launch_resort(pg_pset *ps, cudaStream_t st, int64_t *n_alive);
cudaError_t prepare_resort(pg_pset *ps);
cudaError_t launch_moments(const pg_pset *ps, double *out7, cudaStream_t st);

}  // namespace pg

using namespace pg;

#define CU(call)                                                                      \
  do {                                                                                \
    cudaError_t e_ = (call);                                                          \
    if (e_ != cudaSuccess) {                                                          \
      set_error("%s failed: %s", #call, cudaGetErrorString(e_));                      \
      return e_ == cudaErrorMemoryAllocation ? PG_ERR_NOMEM : PG_ERR_CUDA;            \
    }                                                                                 \
  } while (0)

#define ARG(cond, msg)                                                                \
  do {                                                                                \
    if (!(cond)) {                                                                    \
      set_error("invalid argument: %s", msg);                                         \
      return PG_ERR_ARG;                                                              \
    }                                                                                 \
  } while (0)

namespace {

bool is_device_ptr(const void *p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

bool strictly_increasing(const double *x, int n) {
  for (int i = 0; i < n; ++i)
    if (!std::isfinite(x[i])) return false;
  for (int i = 1; i < n; ++i)
    if (!(x[i] > x[i - 1])) return false;
  return true;
}

// Uniform spacing test: every node within 1e-9 of a spacing of the ideal one.
bool uniform_axis(const std::vector<double> &x, double &x0, double &inv_d) {
  const int n = (int)x.size();
  x0 = x[0];
  if (n < 2) { inv_d = 0.0; return false; }
  const double d = (x[n - 1] - x[0]) / (n - 1);
  for (int i = 0; i < n; ++i)
    if (std::fabs(x[i] - (x[0] + i * d)) > 1e-9 * d) { inv_d = 1.0 / d; return false; }
  inv_d = 1.0 / d;
  return true;
}

__global__ void f64_to_f32_kernel(const double *src, float *dst, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = (float)src[i];
}
__global__ void f32_to_f64_kernel(const float *src, double *dst, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = (double)src[i];
}
__global__ void fill_f64_kernel(double *dst, double v, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = v;
}
__global__ void iota_u64_kernel(uint64_t *dst, uint64_t base, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = base + (uint64_t)i;
}

int grid_for(int64_t n, int sm) {
  int64_t g = (n + 255) / 256;
  const int64_t cap = (int64_t)sm * 16;
  if (g > cap) g = cap;
  return (int)(g < 1 ? 1 : g);
}

// Copy n doubles (host or device) into a device array of the position type.
pg_status upload_coord(const double *src, int64_t n, void *dst, int pos, double fill, int sm,
                       cudaStream_t st) {
  if (n == 0) return PG_OK;
  if (pos == PG_POS_F64) {
    if (src) {
      CU(cudaMemcpyAsync(dst, src, n * 8, cudaMemcpyDefault, st));
    } else {
      fill_f64_kernel<<<grid_for(n, sm), 256, 0, st>>>((double *)dst, fill, n);
      note_launches(1);
      CU(cudaGetLastError());
    }
    return PG_OK;
  }
  if (!src) {
    std::vector<float> h((size_t)n, (float)fill);
    CU(cudaMemcpyAsync(dst, h.data(), n * 4, cudaMemcpyHostToDevice, st));
    CU(cudaStreamSynchronize(st));
    return PG_OK;
  }
  if (!is_device_ptr(src)) {
    // host source: copy the FP64 values to the device (at the copy engines'
    // rate from pinned memory) and round them there
    double *tmp = nullptr;
    CU(dev_alloc((void **)&tmp, (size_t)n * 8));
    cudaError_t e = cudaMemcpyAsync(tmp, src, n * 8, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) {
      f64_to_f32_kernel<<<grid_for(n, sm), 256, 0, st>>>(tmp, (float *)dst, n);
      note_launches(1);
      e = cudaGetLastError();
    }
    const cudaError_t e2 = cudaStreamSynchronize(st);
    dev_free(tmp);
    if (e == cudaSuccess) e = e2;
    if (e != cudaSuccess) {
      set_error("particle upload failed: %s", cudaGetErrorString(e));
      return PG_ERR_CUDA;
    }
    return PG_OK;
  }
  f64_to_f32_kernel<<<grid_for(n, sm), 256, 0, st>>>(src, (float *)dst, n);
  note_launches(1);
  CU(cudaGetLastError());
  return PG_OK;
}

}  // namespace

namespace pg {
pg_status alloc_arrays(PsetArrays &A, int pos, int64_t cap, int nvar) {
  const size_t n = (size_t)std::max<int64_t>(cap, 1);
  cudaError_t e = cudaSuccess;
  auto al = [&](void **p, size_t b) {
    if (e == cudaSuccess) e = dev_alloc(p, b);
  };
  if (pos == PG_POS_CELL) {
    al((void **)&A.ci, n * 4); al((void **)&A.cj, n * 4); al((void **)&A.ck, n * 4);
    al((void **)&A.fx, n * 4); al((void **)&A.fy, n * 4); al((void **)&A.fz, n * 4);
  } else {
    const size_t el = pos_elem(pos);
    al(&A.x, n * el); al(&A.y, n * el); al(&A.z, n * el);
  }
  al((void **)&A.time, n * 8);
  al((void **)&A.id, n * 8);
  al((void **)&A.step, n * 4);
  al((void **)&A.status, n);
  al((void **)&A.age, n * 8);
  al((void **)&A.hstep, n * 8);
  if (nvar > 0) al((void **)&A.var, n * 8 * (size_t)nvar);
  if (e != cudaSuccess) {
    A.free_all();
    cudaGetLastError();
    set_error("device allocation of %lld particles failed: %s", (long long)cap,
              cudaGetErrorString(e));
    return PG_ERR_NOMEM;
  }
  return PG_OK;
}

}  // namespace pg

namespace {

PsetArrays arrays_of(const pg_pset *ps) { return pset_arrays(ps); }
void set_arrays(pg_pset *ps, const PsetArrays &A) { pset_set_arrays(ps, A); }

// The device arrays holding a particle set's state (n entries each from the
// given pointer), with element sizes; variable j starts at var + j * cap.
std::vector<std::pair<void *, size_t>> state_arrays(const PsetArrays &A, int pos, int nvar,
                                                    int64_t cap) {
  std::vector<std::pair<void *, size_t>> v;
  if (pos == PG_POS_CELL) {
    v = {{A.ci, 4}, {A.cj, 4}, {A.ck, 4}, {A.fx, 4}, {A.fy, 4}, {A.fz, 4},
         {A.time, 8}, {A.id, 8}, {A.step, 4}, {A.status, 1}};
  } else {
    const size_t el = pos_elem(pos);
    v = {{A.x, el}, {A.y, el}, {A.z, el}, {A.time, 8}, {A.id, 8}, {A.step, 4}, {A.status, 1}};
  }
  v.push_back({A.age, 8});
  v.push_back({A.hstep, 8});
  for (int j = 0; j < nvar; ++j) v.push_back({A.var ? A.var + (size_t)j * cap : nullptr, 8});
  return v;
}

GridArgs grid_args(const pg_fieldset *fs) {
  GridArgs g;
  g.nx = fs->nx; g.ny = fs->ny; g.nz = fs->nz;
  g.mesh = fs->mesh; g.periodic = fs->periodic;
  g.lon = fs->d_axes64; g.lat = fs->d_axes64 + fs->nx; g.depth = fs->d_axes64 + fs->nx + fs->ny;
  g.lonf = fs->d_axes32; g.latf = fs->d_axes32 + fs->nx; g.depthf = fs->d_axes32 + fs->nx + fs->ny;
  for (int a = 0; a < 3; ++a) {
    g.uni[a] = fs->uni[a];
    g.x0[a] = fs->x0[a];
    g.inv_d[a] = fs->inv_d[a];
    g.x0f[a] = (float)fs->x0[a];
    g.inv_df[a] = (float)fs->inv_d[a];
  }
  g.lon_end = fs->lon[0] + 360.0;
  g.lon_end_f = (float)g.lon_end;
  for (int a = 0; a < 3; ++a) {
    const std::vector<double> &x = a == 0 ? fs->lon : (a == 1 ? fs->lat : fs->depth);
    g.lo[a] = x.front(); g.hi[a] = x.back();
    g.lof[a] = (float)x.front(); g.hif[a] = (float)x.back();
  }
  const double D = 1852.0 * 60.0;
  for (int a = 0; a < 3; ++a) {
    g.d[a] = fs->inv_d[a] != 0.0 ? 1.0 / fs->inv_d[a] : 0.0;
    const std::vector<double> &x = a == 0 ? fs->lon : (a == 1 ? fs->lat : fs->depth);
    if (x.size() > 1) g.d[a] = (x.back() - x.front()) / (double)(x.size() - 1);
    g.df[a] = (float)g.d[a];
    const double metres = (fs->mesh == PG_SPHERICAL && a < 2) ? D * g.d[a] : g.d[a];
    g.inv_m[a] = metres != 0.0 ? (float)(1.0 / metres) : 0.f;
  }
  return g;
}

}  // namespace

GridArgs pg::grid_args_of(const pg_fieldset *fs) { return grid_args(fs); }

PsetArrays pg::pset_arrays(const pg_pset *ps) {
  PsetArrays A;
  A.x = ps->x; A.y = ps->y; A.z = ps->z;
  A.ci = ps->ci; A.cj = ps->cj; A.ck = ps->ck;
  A.fx = ps->fx; A.fy = ps->fy; A.fz = ps->fz;
  A.time = ps->time; A.id = ps->id; A.step = ps->step; A.status = ps->status;
  A.age = ps->age; A.var = ps->var; A.hstep = ps->hstep;
  return A;
}

void pg::pset_set_arrays(pg_pset *ps, const PsetArrays &A) {
  ps->x = A.x; ps->y = A.y; ps->z = A.z;
  ps->ci = A.ci; ps->cj = A.cj; ps->ck = A.ck;
  ps->fx = A.fx; ps->fy = A.fy; ps->fz = A.fz;
  ps->time = A.time; ps->id = A.id; ps->step = A.step; ps->status = A.status;
  ps->age = A.age; ps->var = A.var; ps->hstep = A.hstep;
}

namespace {

// ---------------------------------------------------------------- streaming

// Snapshot index for a (possibly periodic) snapshot counter m: periodic
// fields repeat every nt snapshots.
int snap_of(const pg_fieldset *fs, long long m) {
  const long long nt = fs->nt;
  long long r = m % nt;
  if (r < 0) r += nt;
  return (int)r;
}

// Unwrapped snapshot counter m with T(m) <= t < T(m+1), where
// T(m) = times[m mod nt] + floor(m / nt) * period (periodic) or times[m].
long long snap_counter(const pg_fieldset *fs, double t) {
  const int nt = fs->nt;
  double base = 0.0;
  long long turns = 0;
  double tt = t;
  if (fs->period > 0.0) {
    double r = std::fmod(t - fs->times[0], fs->period);
    if (r < 0.0) r += fs->period;
    turns = (long long)std::floor((t - fs->times[0] - r) / fs->period + 0.5);
    tt = fs->times[0] + r;
    base = (double)turns;
  }
  (void)base;
  int s = (int)(std::upper_bound(fs->times.begin(), fs->times.end(), tt) - fs->times.begin()) - 1;
  if (s < 0) s = 0;
  if (fs->period <= 0.0 && s > nt - 2) s = std::max(0, nt - 2);
  return turns * nt + s;
}

double snap_time(const pg_fieldset *fs, long long m) {
  const long long nt = fs->nt;
  long long q = m >= 0 ? m / nt : -((-m + nt - 1) / nt);
  const int s = (int)(m - q * nt);
  return fs->times[s] + (fs->period > 0.0 ? (double)q * fs->period : 0.0);
}

pg_status upload_to_slot(pg_fieldset *fs, Slot &sl, int s) {
  cudaStream_t side = fs->side;
  CU(cudaStreamWaitEvent(side, sl.free, 0));
  const size_t el = fs->src_dtype == PG_F64 ? 8 : 4;
  const size_t bytes = (size_t)fs->nfields * fs->nodes * el;
  const void *src = nullptr;
  if (fs->cb) {
    CU(cudaEventSynchronize(fs->stage_free));
    if (fs->cb(fs->cb_user, s, fs->h_pinned, bytes) != 0) {
      set_error("snapshot callback failed for snapshot %d", s);
      return PG_ERR_CALLBACK;
    }
    CU(cudaMemcpyAsync(fs->d_stage, fs->h_pinned, bytes, cudaMemcpyHostToDevice, side));
    CU(cudaEventRecord(fs->stage_free, side));
    src = fs->d_stage;
    fs->upload_h2d_bytes += (int64_t)bytes;
  } else {
    const void *p = fs->src_ptrs[s];
    if (is_device_ptr(p)) {
      src = p;
    } else {
      CU(cudaMemcpyAsync(fs->d_stage, p, bytes, cudaMemcpyHostToDevice, side));
      src = fs->d_stage;
      fs->upload_h2d_bytes += (int64_t)bytes;
    }
  }
  ++fs->uploads;
  CU(launch_repack(src, fs->src_dtype, fs->nfields, fs->nodes, sl.buf, fs->storage, sl.scales,
                   fs->d_amax, fs->sm_count, side));
  CU(cudaEventRecord(sl.ready, side));
  sl.s = s;
  return PG_OK;
}

// Make the snapshots `need` resident (uploading the missing ones on the side
// stream), then start uploading the snapshots of `prefetch`, in order, into
// slots no chunk needs now.
pg_status ensure_slots(pg_fieldset *fs, const std::vector<int> &need,
                       const std::vector<int> &prefetch, cudaStream_t st) {
  auto find = [&](int s) {
    for (int q = 0; q < (int)fs->slot.size(); ++q)
      if (fs->slot[q].s == s) return q;
    return -1;
  };
  auto in = [](const std::vector<int> &v, int s, size_t upto) {
    return std::find(v.begin(), v.begin() + (std::ptrdiff_t)std::min(upto, v.size()), s) !=
           v.begin() + (std::ptrdiff_t)std::min(upto, v.size());
  };
  auto needed = [&](int q) { return in(need, fs->slot[q].s, need.size()); };
  for (int s : need) {
    if (find(s) >= 0) continue;
    int q = -1;
    for (int c = 0; c < (int)fs->slot.size() && q < 0; ++c)
      if (!needed(c) && !in(prefetch, fs->slot[c].s, prefetch.size())) q = c;
    for (int c = 0; c < (int)fs->slot.size() && q < 0; ++c)
      if (!needed(c)) q = c;
    if (q < 0) {
      set_error("streamed field needs more resident snapshots per chunk than its ring holds");
      return PG_ERR_UNSUPPORTED;
    }
    pg_status r = upload_to_slot(fs, fs->slot[q], s);
    if (r) return r;
  }
  // device table: resident slots only
  std::vector<const void *> tab((size_t)fs->nt, nullptr);
  for (int s : need) {
    const int q = find(s);
    CU(cudaStreamWaitEvent(st, fs->slot[q].ready, 0));
    tab[s] = fs->slot[q].buf;
    CU(cudaMemcpyAsync(fs->d_scales + (size_t)s * fs->nfields, fs->slot[q].scales,
                       sizeof(float) * fs->nfields, cudaMemcpyDeviceToDevice, st));
  }
  CU(cudaMemcpyAsync(fs->d_tab, tab.data(), sizeof(void *) * fs->nt, cudaMemcpyHostToDevice, st));
  for (size_t i = 0; i < prefetch.size(); ++i) {
    const int s = prefetch[i];
    if (find(s) >= 0) continue;
    // a slot holding neither a needed snapshot nor an earlier prefetch
    int q = -1;
    for (int c = 0; c < (int)fs->slot.size() && q < 0; ++c)
      if (!needed(c) && !in(prefetch, fs->slot[c].s, i)) q = c;
    if (q < 0) break;
    pg_status r = upload_to_slot(fs, fs->slot[q], s);
    if (r) return r;
  }
  return PG_OK;
}

void mark_slots_used(pg_fieldset *fs, const std::vector<int> &need, cudaStream_t st) {
  for (int q = 0; q < (int)fs->slot.size(); ++q)
    if (std::find(need.begin(), need.end(), fs->slot[q].s) != need.end())
      cudaEventRecord(fs->slot[q].free, st);
}

void free_streaming(pg_fieldset *fs) {
  for (auto &sl : fs->slot) {
    dev_free(sl.buf);
    dev_free(sl.scales);
    if (sl.ready) cudaEventDestroy(sl.ready);
    if (sl.free) cudaEventDestroy(sl.free);
    sl = Slot();
  }
  if (fs->h_pinned) cudaFreeHost(fs->h_pinned);
  fs->h_pinned = nullptr;
  if (fs->side) cudaStreamDestroy(fs->side);
  fs->side = nullptr;
  if (fs->stage_free) cudaEventDestroy(fs->stage_free);
  fs->stage_free = nullptr;
  fs->streaming = false;
  fs->cb = nullptr;
  fs->src_ptrs.clear();
}

void free_resident(pg_fieldset *fs) {
  for (void *p : fs->slabs) dev_free(p);
  fs->slabs.clear();
}

void free_tracers(pg_fieldset *fs) {
  for (void *p : fs->tr_slabs) dev_free(p);
  fs->tr_slabs.assign(fs->tr_slabs.size(), nullptr);
}

// Initial variables of particles [off, off + n): age 0, sampled values NaN
// (nothing sampled yet).
pg_status init_variables(pg_pset *ps, int64_t off, int64_t n, cudaStream_t st) {
  if (n <= 0) return PG_OK;
  const int sm = ps->fs->sm_count;
  fill_f64_kernel<<<grid_for(n, sm), 256, 0, st>>>(ps->age + off, 0.0, n);
  fill_f64_kernel<<<grid_for(n, sm), 256, 0, st>>>(ps->hstep + off, 0.0, n);
  note_launches(2);
  for (int j = 0; j < ps->nvar; ++j) {
    fill_f64_kernel<<<grid_for(n, sm), 256, 0, st>>>(ps->var + (size_t)j * ps->cap + off,
                                                     std::numeric_limits<double>::quiet_NaN(), n);
    note_launches(1);
  }
  CU(cudaGetLastError());
  CU(cudaStreamSynchronize(st));
  return PG_OK;
}

}  // namespace

namespace pg {

// The kernel argument block of kernel k on field set fs: parameters given as
// NaN, and those of the worked example's behaviours, come from the field
// set's constants ("Kh", "w_sink", "dwelling_depth", "max_age").
pg_status resolve_kernel(const pg_kernel *k, const pg_fieldset *fs, uint64_t seed, KernArgs &a) {
  auto constant = [&](const char *name, double &v) -> bool {
    auto it = fs->constants.find(name);
    if (it == fs->constants.end()) {
      set_error("the kernel needs the field set constant \"%s\"", name);
      return false;
    }
    v = it->second;
    return true;
  };
  a = KernArgs();
  a.scheme = k->scheme; a.beh = k->beh;
  a.kh = k->kh; a.w_sink = k->w_sink;
  if ((k->beh & PG_BROWNIAN) && std::isnan(a.kh) && !constant("Kh", a.kh)) return PG_ERR_STATE;
  if ((k->beh & (PG_SINK | PG_SETTLE)) && std::isnan(a.w_sink) && !constant("w_sink", a.w_sink))
    return PG_ERR_STATE;
  if (std::isnan(a.kh)) a.kh = 0.0;
  if (std::isnan(a.w_sink)) a.w_sink = 0.0;
  if ((k->beh & PG_SETTLE) && !constant("dwelling_depth", a.dwell)) return PG_ERR_STATE;
  if ((k->beh & PG_AGE) && !constant("max_age", a.max_age)) return PG_ERR_STATE;
  if (k->scheme == PG_RKF45) {
    if (!constant("rkf45_tol", a.rk_tol)) return PG_ERR_STATE;
    auto lo = fs->constants.find("rkf45_min_dt"), hi = fs->constants.find("rkf45_max_dt");
    a.rk_hmin = lo != fs->constants.end() ? lo->second : 1.0;
    a.rk_hmax = hi != fs->constants.end() ? hi->second : 0.0;   // 0: the execute's |dt|
    if (!(a.rk_tol > 0.0) || !(a.rk_hmin > 0.0) || a.rk_hmax < 0.0) {
      set_error("RKF45 needs rkf45_tol > 0, rkf45_min_dt > 0, rkf45_max_dt >= 0");
      return PG_ERR_ARG;
    }
  }
  if (!(a.kh >= 0.0)) {
    set_error("Kh must be >= 0");
    return PG_ERR_ARG;
  }
  a.seed = seed; a.deg_m = 1852.0 * 60.0;
  a.deg_m_f = (float)a.deg_m; a.inv_deg_m_f = (float)(1.0 / a.deg_m);
  a.kh_f = (float)a.kh; a.w_sink_f = (float)a.w_sink;
  a.dwell_f = (float)a.dwell;
  return PG_OK;
}

}  // namespace pg

// ======================================================================== ABI

extern "C" {

const char *pg_last_error(void) { return g_err.c_str(); }

const char *pg_version(void) { return "parcels-gb300 0.1 (sm_103a)"; }

pg_status pg_debug_set_alloc_limit(int64_t bytes) {
  g_alloc_limit = bytes < 0 ? -1 : g_alloc_bytes + bytes;
  return PG_OK;
}

pg_status pg_fieldset_create(const pg_grid *grid, int mesh, int periodic_lon, int nfields,
                             int storage, pg_fieldset **out) {
  clear_error();
  ARG(grid && out, "grid and out must not be NULL");
  ARG(grid->nx >= 2 && grid->ny >= 2 && grid->nz >= 1, "need nx >= 2, ny >= 2, nz >= 1");
  ARG(grid->lon && grid->lat && (grid->nz == 1 || grid->depth), "axis pointers must be set");
  ARG(strictly_increasing(grid->lon, grid->nx), "lon must be finite and strictly increasing");
  ARG(strictly_increasing(grid->lat, grid->ny), "lat must be finite and strictly increasing");
  ARG(grid->nz == 1 || strictly_increasing(grid->depth, grid->nz),
      "depth must be finite and strictly increasing");
  ARG(mesh == PG_FLAT || mesh == PG_SPHERICAL, "mesh must be PG_FLAT or PG_SPHERICAL");
  ARG(!periodic_lon || mesh == PG_SPHERICAL, "periodic lon needs a spherical mesh");
  ARG(!periodic_lon || grid->lon[grid->nx - 1] - grid->lon[0] < 360.0,
      "periodic lon axis must span less than 360 degrees");
  ARG(nfields == 2 || (nfields == 3 && grid->nz > 1), "nfields must be 2, or 3 with nz > 1");
  ARG(storage >= PG_F64 && storage <= PG_BF16S, "unknown storage");
  auto *fs = new pg_fieldset();
  CU(cudaGetDevice(&fs->device));
  CU(cudaDeviceGetAttribute(&fs->sm_count, cudaDevAttrMultiProcessorCount, fs->device));
  fs->nx = grid->nx; fs->ny = grid->ny; fs->nz = grid->nz;
  fs->mesh = mesh; fs->periodic = periodic_lon ? 1 : 0;
  fs->nfields = nfields; fs->storage = storage;
  fs->lon.assign(grid->lon, grid->lon + grid->nx);
  fs->lat.assign(grid->lat, grid->lat + grid->ny);
  if (grid->nz > 1) fs->depth.assign(grid->depth, grid->depth + grid->nz);
  else fs->depth.assign(1, grid->depth ? grid->depth[0] : 0.0);
  fs->uni[0] = uniform_axis(fs->lon, fs->x0[0], fs->inv_d[0]);
  fs->uni[1] = uniform_axis(fs->lat, fs->x0[1], fs->inv_d[1]);
  fs->uni[2] = grid->nz > 1 ? uniform_axis(fs->depth, fs->x0[2], fs->inv_d[2]) : 0;
  fs->nodes = (size_t)fs->nx * fs->ny * fs->nz;
  fs->slab_bytes = fs->nodes * (nfields == 2 ? 2 : 4) * storage_elem(storage);
  const int na = fs->nx + fs->ny + fs->nz;
  std::vector<double> ax;
  ax.insert(ax.end(), fs->lon.begin(), fs->lon.end());
  ax.insert(ax.end(), fs->lat.begin(), fs->lat.end());
  ax.insert(ax.end(), fs->depth.begin(), fs->depth.end());
  std::vector<float> axf(ax.begin(), ax.end());
  cudaError_t e = dev_alloc((void **)&fs->d_axes64, na * 8);
  if (e == cudaSuccess) e = dev_alloc((void **)&fs->d_axes32, na * 4);
  if (e == cudaSuccess) e = dev_alloc((void **)&fs->d_amax, 4 * sizeof(unsigned));
  if (e == cudaSuccess) e = cudaMemcpy(fs->d_axes64, ax.data(), na * 8, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(fs->d_axes32, axf.data(), na * 4, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    dev_free(fs->d_axes64); dev_free(fs->d_axes32); dev_free(fs->d_amax);
    delete fs;
    cudaGetLastError();
    set_error("field set allocation failed: %s", cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? PG_ERR_NOMEM : PG_ERR_CUDA;
  }
  *out = fs;
  return PG_OK;
}

pg_status pg_fieldset_set_times(pg_fieldset *fs, int nt, const double *times, double period) {
  clear_error();
  ARG(fs && times && nt >= 1, "need a field set and nt >= 1 times");
  ARG(strictly_increasing(times, nt), "times must be finite and strictly increasing");
  ARG(std::isfinite(period) && period >= 0.0, "period must be >= 0");
  ARG(period == 0.0 || (nt >= 2 && period > times[nt - 1] - times[0]),
      "a periodic field needs nt >= 2 and period > times[nt-1] - times[0]");
  ARG(!fs->streaming, "set the times before streaming is configured");
  double *d_times = nullptr;
  const void **d_tab = nullptr;
  float *d_scales = nullptr;
  const void **d_ttab = nullptr;
  cudaError_t e = dev_alloc((void **)&d_times, nt * 8);
  if (e == cudaSuccess) e = dev_alloc((void **)&d_tab, nt * sizeof(void *));
  if (e == cudaSuccess) e = dev_alloc((void **)&d_scales, (size_t)nt * fs->nfields * 4);
  if (e == cudaSuccess) e = dev_alloc((void **)&d_ttab, 2 * (size_t)nt * sizeof(void *));
  std::vector<float> ones((size_t)nt * fs->nfields, 1.0f);
  std::vector<const void *> nulls((size_t)nt, nullptr);
  if (e == cudaSuccess) e = cudaMemcpy(d_times, times, nt * 8, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(d_tab, nulls.data(), nt * sizeof(void *), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(d_scales, ones.data(), ones.size() * 4, cudaMemcpyHostToDevice);
  std::vector<const void *> tnulls(2 * (size_t)nt, nullptr);
  if (e == cudaSuccess)
    e = cudaMemcpy(d_ttab, tnulls.data(), tnulls.size() * sizeof(void *), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    dev_free(d_times); dev_free(d_tab); dev_free(d_scales); dev_free(d_ttab);
    cudaGetLastError();
    set_error("allocation for %d snapshots failed: %s", nt, cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? PG_ERR_NOMEM : PG_ERR_CUDA;
  }
  free_resident(fs);
  free_tracers(fs);
  dev_free(fs->d_times); dev_free(fs->d_tab); dev_free(fs->d_scales); dev_free(fs->d_ttab);
  fs->d_times = d_times; fs->d_tab = d_tab; fs->d_scales = d_scales; fs->d_ttab = d_ttab;
  fs->tr_slabs.assign(2 * (size_t)nt, nullptr);
  fs->nt = nt;
  fs->times.assign(times, times + nt);
  fs->period = period;
  fs->slabs.assign((size_t)nt, nullptr);
  fs->h_scales = ones;
  return PG_OK;
}

pg_status pg_fieldset_load_snapshot(pg_fieldset *fs, int s, const void *data, int src_dtype,
                                    void *stream) {
  clear_error();
  ARG(fs && data, "field set and data must not be NULL");
  ARG(fs->nt > 0, "set the snapshot times first");
  ARG(s >= 0 && s < fs->nt, "snapshot index out of range");
  ARG(src_dtype == PG_F64 || src_dtype == PG_F32, "src_dtype must be PG_F64 or PG_F32");
  ARG(!fs->streaming, "field set is streamed; snapshots are not resident");
  cudaStream_t st = (cudaStream_t)stream;
  void *slab = fs->slabs[s];
  bool fresh = false;
  if (!slab) {
    CU(dev_alloc(&slab, fs->slab_bytes));
    fresh = true;
  }
  const void *src = data;
  const size_t el = src_dtype == PG_F64 ? 8 : 4;
  const size_t bytes = (size_t)fs->nfields * fs->nodes * el;
  if (!is_device_ptr(data)) {
    if (fs->stage_bytes < bytes) {
      dev_free(fs->d_stage);
      fs->d_stage = nullptr;
      fs->stage_bytes = 0;
      cudaError_t e = dev_alloc(&fs->d_stage, bytes);
      if (e != cudaSuccess) {
        if (fresh) dev_free(slab);
        cudaGetLastError();
        set_error("staging allocation failed: %s", cudaGetErrorString(e));
        return PG_ERR_NOMEM;
      }
      fs->stage_bytes = bytes;
    }
    CU(cudaMemcpyAsync(fs->d_stage, data, bytes, cudaMemcpyDefault, st));
    src = fs->d_stage;
  }
  float *scales = fs->d_scales + (size_t)s * fs->nfields;
  CU(launch_repack(src, src_dtype, fs->nfields, fs->nodes, slab, fs->storage, scales, fs->d_amax,
                   fs->sm_count, st));
  CU(cudaMemcpyAsync(fs->h_scales.data() + (size_t)s * fs->nfields, scales,
                     sizeof(float) * fs->nfields, cudaMemcpyDeviceToHost, st));
  const void *entry = slab;
  CU(cudaMemcpyAsync(fs->d_tab + s, &entry, sizeof(void *), cudaMemcpyHostToDevice, st));
  CU(cudaStreamSynchronize(st));
  fs->slabs[s] = slab;
  return PG_OK;
}

pg_status pg_fieldset_stream(pg_fieldset *fs, const void *const *ptrs, pg_snapshot_cb cb,
                             void *user, int src_dtype) {
  clear_error();
  ARG(fs, "field set must not be NULL");
  ARG(fs->nt > 0, "set the snapshot times first");
  ARG((ptrs != nullptr) != (cb != nullptr), "exactly one of ptrs and cb must be given");
  ARG(src_dtype == PG_F64 || src_dtype == PG_F32, "src_dtype must be PG_F64 or PG_F32");
  if (ptrs)
    for (int s = 0; s < fs->nt; ++s) ARG(ptrs[s] != nullptr, "every snapshot pointer must be set");
  const size_t el = src_dtype == PG_F64 ? 8 : 4;
  const size_t bytes = (size_t)fs->nfields * fs->nodes * el;
  // everything new is allocated first; the field set changes only once all
  // of it is in place (a failure leaves it as it was)
  std::vector<Slot> ring(fs->slot.size());
  void *stage = nullptr, *pinned = nullptr;
  cudaStream_t side = nullptr;
  cudaEvent_t stage_free = nullptr;
  cudaError_t e = cudaSuccess;
  for (auto &sl : ring) {
    if (e == cudaSuccess) e = dev_alloc(&sl.buf, fs->slab_bytes);
    if (e == cudaSuccess) e = dev_alloc((void **)&sl.scales, 4 * sizeof(float));
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sl.ready, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sl.free, cudaEventDisableTiming);
    sl.s = -1;
  }
  if (e == cudaSuccess && fs->stage_bytes < bytes) e = dev_alloc(&stage, bytes);
  if (e == cudaSuccess && cb) e = cudaMallocHost(&pinned, bytes);
  // the side stream at the highest priority: its repack kernel then takes
  // SM slots as the advection kernel's blocks retire, instead of waiting
  // for the whole launch, and the next copy into the staging buffer follows
  int prio_lo = 0, prio_hi = 0;
  if (e == cudaSuccess) e = cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi);
  if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&side, cudaStreamNonBlocking, prio_hi);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&stage_free, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventRecord(stage_free, side);
  if (e != cudaSuccess) {
    for (auto &sl : ring) {
      dev_free(sl.buf);
      dev_free(sl.scales);
      if (sl.ready) cudaEventDestroy(sl.ready);
      if (sl.free) cudaEventDestroy(sl.free);
    }
    dev_free(stage);
    if (pinned) cudaFreeHost(pinned);
    if (side) cudaStreamDestroy(side);
    if (stage_free) cudaEventDestroy(stage_free);
    cudaGetLastError();
    set_error("streaming setup failed: %s", cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? PG_ERR_NOMEM : PG_ERR_CUDA;
  }
  free_streaming(fs);
  free_resident(fs);
  fs->slabs.assign((size_t)fs->nt, nullptr);
  fs->slot = ring;
  if (stage) {
    dev_free(fs->d_stage);
    fs->d_stage = stage;
    fs->stage_bytes = bytes;
  }
  fs->h_pinned = pinned;
  fs->side = side;
  fs->stage_free = stage_free;
  fs->streaming = true;
  fs->cb = cb;
  fs->cb_user = user;
  fs->src_dtype = src_dtype;
  if (ptrs) fs->src_ptrs.assign(ptrs, ptrs + fs->nt);
  return PG_OK;
}

pg_status pg_fieldset_set_ring(pg_fieldset *fs, int slots) {
  clear_error();
  ARG(fs, "field set must not be NULL");
  ARG(slots >= 4 && slots <= 64, "the ring holds 4 to 64 snapshots");
  ARG(!fs->streaming, "set the ring size before pg_fieldset_stream");
  fs->slot.assign((size_t)slots, Slot());
  return PG_OK;
}

pg_status pg_fieldset_device_bytes(const pg_fieldset *fs, size_t *bytes) {
  clear_error();
  ARG(fs && bytes, "arguments must not be NULL");
  size_t b = 0;
  for (void *p : fs->slabs) b += p ? fs->slab_bytes : 0;
  if (fs->streaming) b += fs->slot.size() * fs->slab_bytes;
  *bytes = b;
  return PG_OK;
}

pg_status pg_fieldset_stats(pg_fieldset *fs, int reset, int64_t *uploads, int64_t *h2d_bytes) {
  clear_error();
  ARG(fs, "field set must not be NULL");
  if (uploads) *uploads = fs->uploads;
  if (h2d_bytes) *h2d_bytes = fs->upload_h2d_bytes;
  if (reset) { fs->uploads = 0; fs->upload_h2d_bytes = 0; }
  return PG_OK;
}

pg_status pg_fieldset_get_scale(const pg_fieldset *fs, int s, int f, float *scale) {
  clear_error();
  ARG(fs && scale, "arguments must not be NULL");
  ARG(s >= 0 && s < fs->nt && f >= 0 && f < fs->nfields, "index out of range");
  ARG(!fs->streaming, "scales of streamed snapshots are not kept");
  *scale = fs->h_scales[(size_t)s * fs->nfields + f];
  return PG_OK;
}

pg_status pg_fieldset_add_constant(pg_fieldset *fs, const char *name, double value) {
  clear_error();
  ARG(fs && name && name[0], "field set and a non-empty name are needed");
  ARG(std::isfinite(value), "constants must be finite");
  fs->constants[name] = value;
  return PG_OK;
}

pg_status pg_fieldset_get_constant(const pg_fieldset *fs, const char *name, double *value) {
  clear_error();
  ARG(fs && name && value, "arguments must not be NULL");
  auto it = fs->constants.find(name);
  if (it == fs->constants.end()) {
    set_error("the field set has no constant \"%s\"", name);
    return PG_ERR_ARG;
  }
  *value = it->second;
  return PG_OK;
}

pg_status pg_fieldset_set_interp(pg_fieldset *fs, int method) {
  clear_error();
  ARG(fs, "field set must not be NULL");
  ARG(method == PG_LINEAR || method == PG_NEAREST, "method must be PG_LINEAR or PG_NEAREST");
  fs->interp = method;
  return PG_OK;
}

pg_status pg_fieldset_add_scalar(pg_fieldset *fs, const char *name, int method, int *index) {
  clear_error();
  ARG(fs && name && name[0], "field set and a non-empty name are needed");
  ARG(method == PG_LINEAR || method == PG_NEAREST, "method must be PG_LINEAR or PG_NEAREST");
  ARG(fs->nt > 0, "set the snapshot times first");
  if (fs->ntr >= 2) {
    set_error("a field set holds at most two scalar fields");
    return PG_ERR_UNSUPPORTED;
  }
  const int q = fs->ntr;
  fs->tr_name[q] = name;
  fs->tr_interp[q] = method;
  fs->ntr = q + 1;
  if (index) *index = q;
  return PG_OK;
}

pg_status pg_fieldset_load_scalar(pg_fieldset *fs, int index, int s, const void *data,
                                  int src_dtype, void *stream) {
  clear_error();
  ARG(fs && data, "field set and data must not be NULL");
  ARG(index >= 0 && index < fs->ntr, "no scalar field of that index");
  ARG(s >= 0 && s < fs->nt, "snapshot index out of range");
  ARG(src_dtype == PG_F64 || src_dtype == PG_F32, "src_dtype must be PG_F64 or PG_F32");
  cudaStream_t st = (cudaStream_t)stream;
  const size_t el = fs->storage == PG_F64 ? 8 : 4;
  void *&slab = fs->tr_slabs[(size_t)index * fs->nt + s];
  void *fresh = nullptr;
  if (!slab) CU(dev_alloc(&fresh, fs->nodes * el));
  void *dst = slab ? slab : fresh;
  const size_t src_el = src_dtype == PG_F64 ? 8 : 4;
  cudaError_t e = cudaSuccess;
  if (src_el == el) {
    e = cudaMemcpyAsync(dst, data, fs->nodes * el, cudaMemcpyDefault, st);
  } else {
    // convert on the host side of the copy: FP64 source to FP32 storage, or
    // FP32 source to FP64 storage (exact)
    void *tmp = nullptr;
    e = dev_alloc(&tmp, fs->nodes * src_el);
    if (e == cudaSuccess) e = cudaMemcpyAsync(tmp, data, fs->nodes * src_el, cudaMemcpyDefault, st);
    if (e == cudaSuccess) {
      if (src_el == 8) f64_to_f32_kernel<<<grid_for((int64_t)fs->nodes, fs->sm_count), 256, 0, st>>>(
          (const double *)tmp, (float *)dst, (int64_t)fs->nodes);
      else f32_to_f64_kernel<<<grid_for((int64_t)fs->nodes, fs->sm_count), 256, 0, st>>>(
          (const float *)tmp, (double *)dst, (int64_t)fs->nodes);
      note_launches(1);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    dev_free(tmp);
  }
  const void *entry = dst;
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(fs->d_ttab + (size_t)index * fs->nt + s, &entry, sizeof(void *),
                        cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    dev_free(fresh);
    cudaGetLastError();
    set_error("loading scalar field %d, snapshot %d failed: %s", index, s, cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? PG_ERR_NOMEM : PG_ERR_CUDA;
  }
  slab = dst;
  return PG_OK;
}

pg_status pg_fieldset_destroy(pg_fieldset *fs) {
  clear_error();
  if (!fs) return PG_OK;
  cudaDeviceSynchronize();
  free_streaming(fs);
  free_resident(fs);
  free_tracers(fs);
  dev_free(fs->d_axes64); dev_free(fs->d_axes32); dev_free(fs->d_amax);
  dev_free(fs->d_times); dev_free(fs->d_tab); dev_free(fs->d_scales); dev_free(fs->d_stage);
  dev_free(fs->d_ttab);
  delete fs;
  return PG_OK;
}

pg_status pg_kernel_create(int scheme, unsigned behaviours, double kh, double w_sink,
                           pg_kernel **out) {
  clear_error();
  ARG(out, "out must not be NULL");
  ARG(scheme == PG_EULER || scheme == PG_RK4 || scheme == PG_RKF45,
      "scheme must be PG_EULER, PG_RK4 or PG_RKF45");
  ARG((behaviours & ~(PG_BROWNIAN | PG_SINK | PG_SETTLE | PG_AGE | PG_SAMPLE)) == 0,
      "unknown behaviour bits");
  ARG(std::isnan(kh) || (std::isfinite(kh) && kh >= 0.0), "kh must be NaN, or finite and >= 0");
  ARG(std::isnan(w_sink) || std::isfinite(w_sink), "w_sink must be NaN or finite");
  auto *k = new pg_kernel();
  k->scheme = scheme; k->beh = behaviours; k->kh = kh; k->w_sink = w_sink;
  *out = k;
  return PG_OK;
}

pg_status pg_kernel_destroy(pg_kernel *k) {
  delete k;
  return PG_OK;
}

static pg_status fill_particles(pg_pset *ps, int64_t off, int64_t n, const double *lon,
                                const double *lat, const double *depth, const double *time,
                                double t0, const uint64_t *ids, uint64_t id_base,
                                cudaStream_t st, double &tmin, double &tmax) {
  const int sm = ps->fs->sm_count;
  pg_status r;
  if (ps->pos == PG_POS_CELL) {
    // FP64 positions on the device, then split into cell index + offset
    double *tmp = nullptr;
    CU(dev_alloc((void **)&tmp, (size_t)n * 8 * 3));
    r = upload_coord(lon, n, tmp, PG_POS_F64, 0.0, sm, st);
    if (!r) r = upload_coord(lat, n, tmp + n, PG_POS_F64, 0.0, sm, st);
    if (!r) r = upload_coord(depth, n, tmp + 2 * n, PG_POS_F64, ps->fs->depth[0], sm, st);
    if (!r) {
      cudaError_t e = launch_to_cell(grid_args(ps->fs), tmp, tmp + n, tmp + 2 * n, ps->ci + off,
                                     ps->cj + off, ps->ck + off, ps->fx + off, ps->fy + off,
                                     ps->fz + off, n, sm, st);
      if (e == cudaSuccess) e = cudaStreamSynchronize(st);
      if (e != cudaSuccess) {
        set_error("cell conversion failed: %s", cudaGetErrorString(e));
        r = PG_ERR_CUDA;
      }
    }
    dev_free(tmp);
    if (r) return r;
  } else {
    const size_t el = pos_elem(ps->pos);
    if ((r = upload_coord(lon, n, (char *)ps->x + off * el, ps->pos, 0.0, sm, st))) return r;
    if ((r = upload_coord(lat, n, (char *)ps->y + off * el, ps->pos, 0.0, sm, st))) return r;
    if ((r = upload_coord(depth, n, (char *)ps->z + off * el, ps->pos, 0.0, sm, st))) return r;
  }
  tmin = t0; tmax = t0;
  if (time) {
    CU(cudaMemcpyAsync(ps->time + off, time, n * 8, cudaMemcpyDefault, st));
    std::vector<double> h((size_t)n);
    CU(cudaMemcpyAsync(h.data(), time, n * 8, cudaMemcpyDefault, st));
    CU(cudaStreamSynchronize(st));
    tmin = std::numeric_limits<double>::infinity();
    tmax = -tmin;
    for (double v : h) {
      if (!std::isfinite(v)) {
        set_error("particle times must be finite");
        return PG_ERR_ARG;
      }
      tmin = std::min(tmin, v);
      tmax = std::max(tmax, v);
    }
  } else {
    fill_f64_kernel<<<grid_for(n, sm), 256, 0, st>>>(ps->time + off, t0, n);
    note_launches(1);
    CU(cudaGetLastError());
  }
  if (ids) {
    CU(cudaMemcpyAsync(ps->id + off, ids, n * 8, cudaMemcpyDefault, st));
  } else {
    iota_u64_kernel<<<grid_for(n, sm), 256, 0, st>>>(ps->id + off, id_base, n);
    note_launches(1);
    CU(cudaGetLastError());
  }
  CU(cudaMemsetAsync(ps->step + off, 0, n * 4, st));
  CU(cudaMemsetAsync(ps->status + off, 0, n, st));
  CU(cudaStreamSynchronize(st));
  return PG_OK;
}

pg_status pg_pset_create(pg_fieldset *fs, int64_t n, const double *lon, const double *lat,
                         const double *depth, const double *time, double t0,
                         const uint64_t *ids, uint64_t id_base, int pos, uint64_t seed,
                         pg_pset **out) {
  clear_error();
  ARG(fs && out, "field set and out must not be NULL");
  ARG(n >= 0, "n must be >= 0");
  ARG(n == 0 || (lon && lat), "lon and lat must be given");
  ARG(pos == PG_POS_F64 || pos == PG_POS_F32 || pos == PG_POS_CELL,
      "pos must be PG_POS_F64, PG_POS_F32 or PG_POS_CELL");
  ARG(std::isfinite(t0), "t0 must be finite");
  ARG(!(pos != PG_POS_F64 && fs->storage == PG_F64),
      "FP32 or cell positions need FP32/FP16/BF16 storage");
  if (pos == PG_POS_CELL && !(fs->uni[0] && fs->uni[1] && (fs->nz == 1 || fs->uni[2]))) {
    set_error("cell positions need uniformly spaced axes");
    return PG_ERR_UNSUPPORTED;
  }
  auto *ps = new pg_pset();
  ps->fs = fs; ps->pos = pos; ps->seed = seed;
  ps->nvar = fs->ntr;
  PsetArrays A;
  pg_status r = alloc_arrays(A, pos, n, ps->nvar);
  if (r) { delete ps; return r; }
  set_arrays(ps, A);
  ps->cap = std::max<int64_t>(n, 1);
  cudaError_t e = dev_alloc((void **)&ps->d_counter, 8);
  if (e == cudaSuccess) e = dev_alloc((void **)&ps->d_err, 4);
  if (e == cudaSuccess) e = cudaMemset(ps->d_err, 0, 4);
  if (e != cudaSuccess) {
    A.free_all(); dev_free(ps->d_counter); dev_free(ps->d_err);
    delete ps;
    cudaGetLastError();
    set_error("allocation failed: %s", cudaGetErrorString(e));
    return PG_ERR_NOMEM;
  }
  double tmin = t0, tmax = t0;
  if (n > 0) r = fill_particles(ps, 0, n, lon, lat, depth, time, t0, ids, id_base, 0, tmin, tmax);
  if (!r) r = init_variables(ps, 0, n, 0);
  if (r) {
    A.free_all(); dev_free(ps->d_counter); dev_free(ps->d_err);
    delete ps;
    return r;
  }
  ps->n = n;
  ps->t_min = tmin; ps->t_max = tmax;
  *out = ps;
  return PG_OK;
}

pg_status pg_pset_add(pg_pset *ps, int64_t n, const double *lon, const double *lat,
                      const double *depth, const double *time, double t0, const uint64_t *ids,
                      uint64_t id_base) {
  clear_error();
  ARG(ps, "particle set must not be NULL");
  ARG(n >= 0, "n must be >= 0");
  if (n == 0) return PG_OK;
  ARG(lon && lat, "lon and lat must be given");
  ARG(std::isfinite(t0), "t0 must be finite");
  if (ps->n + n > ps->cap) {
    const int64_t cap = std::max<int64_t>(ps->n + n, ps->cap + ps->cap / 2);
    PsetArrays B;
    pg_status r = alloc_arrays(B, ps->pos, cap, ps->nvar);
    if (r) return r;
    PsetArrays A = arrays_of(ps);
    const size_t el = pos_elem(ps->pos);
    const int64_t m = ps->n;
    cudaError_t e = cudaSuccess;
    auto cp = [&](void *d, const void *s, size_t b) {
      if (e == cudaSuccess && b) e = cudaMemcpy(d, s, b, cudaMemcpyDeviceToDevice);
    };
    if (ps->pos == PG_POS_CELL) {
      cp(B.ci, A.ci, m * 4); cp(B.cj, A.cj, m * 4); cp(B.ck, A.ck, m * 4);
      cp(B.fx, A.fx, m * 4); cp(B.fy, A.fy, m * 4); cp(B.fz, A.fz, m * 4);
    } else {
      cp(B.x, A.x, m * el); cp(B.y, A.y, m * el); cp(B.z, A.z, m * el);
    }
    cp(B.time, A.time, m * 8); cp(B.id, A.id, m * 8); cp(B.step, A.step, m * 4);
    cp(B.status, A.status, m);
    cp(B.age, A.age, m * 8);
    cp(B.hstep, A.hstep, m * 8);
    for (int j = 0; j < ps->nvar; ++j)
      cp(B.var + (size_t)j * cap, A.var + (size_t)j * ps->cap, m * 8);
    if (e != cudaSuccess) {
      B.free_all();
      set_error("grow copy failed: %s", cudaGetErrorString(e));
      return PG_ERR_CUDA;
    }
    A.free_all();
    set_arrays(ps, B);
    ps->cap = cap;
  }
  double tmin, tmax;
  pg_status r = fill_particles(ps, ps->n, n, lon, lat, depth, time, t0, ids, id_base, 0, tmin, tmax);
  if (!r) r = init_variables(ps, ps->n, n, 0);
  if (r) return r;
  if (ps->n == 0) { ps->t_min = tmin; ps->t_max = tmax; }
  else { ps->t_min = std::min(ps->t_min, tmin); ps->t_max = std::max(ps->t_max, tmax); }
  ps->n += n;
  return PG_OK;
}

pg_status pg_pset_size(const pg_pset *ps, int64_t *n, int64_t *n_alive) {
  clear_error();
  ARG(ps, "particle set must not be NULL");
  if (n) *n = ps->n;
  if (n_alive) {
    std::vector<uint8_t> h((size_t)ps->n);
    if (ps->n) CU(cudaMemcpy(h.data(), ps->status, ps->n, cudaMemcpyDeviceToHost));
    int64_t a = 0;
    for (uint8_t v : h) a += v == 0;
    *n_alive = a;
  }
  return PG_OK;
}

pg_status pg_pset_get(const pg_pset *ps, double *lon, double *lat, double *depth, double *time,
                      uint64_t *ids, uint32_t *steps, uint8_t *status, void *stream) {
  clear_error();
  ARG(ps, "particle set must not be NULL");
  cudaStream_t st = (cudaStream_t)stream;
  const int64_t n = ps->n;
  if (n == 0) return PG_OK;
  double *tmp = nullptr;
  if (ps->pos == PG_POS_CELL && (lon || lat || depth)) {
    CU(dev_alloc((void **)&tmp, n * 8 * 3));
    cudaError_t e = launch_from_cell(grid_args(ps->fs), ps->ci, ps->cj, ps->ck, ps->fx, ps->fy,
                                     ps->fz, tmp, tmp + n, tmp + 2 * n, n, ps->fs->sm_count, st);
    if (e == cudaSuccess && lon) e = cudaMemcpyAsync(lon, tmp, n * 8, cudaMemcpyDefault, st);
    if (e == cudaSuccess && lat) e = cudaMemcpyAsync(lat, tmp + n, n * 8, cudaMemcpyDefault, st);
    if (e == cudaSuccess && depth) e = cudaMemcpyAsync(depth, tmp + 2 * n, n * 8, cudaMemcpyDefault, st);
    if (e != cudaSuccess) {
      cudaStreamSynchronize(st);
      dev_free(tmp);
      set_error("copy failed: %s", cudaGetErrorString(e));
      return PG_ERR_CUDA;
    }
    lon = lat = depth = nullptr;
  }
  if (ps->pos == PG_POS_F32 && (lon || lat || depth)) CU(dev_alloc((void **)&tmp, n * 8));
  auto coord = [&](void *src, double *dst) -> pg_status {
    if (!dst) return PG_OK;
    if (ps->pos == PG_POS_F64) {
      CU(cudaMemcpyAsync(dst, src, n * 8, cudaMemcpyDefault, st));
    } else {
      f32_to_f64_kernel<<<grid_for(n, ps->fs->sm_count), 256, 0, st>>>((const float *)src, tmp, n);
      note_launches(1);
      CU(cudaGetLastError());
      CU(cudaMemcpyAsync(dst, tmp, n * 8, cudaMemcpyDefault, st));
    }
    return PG_OK;
  };
  pg_status r = PG_OK;
  if (!r) r = coord(ps->x, lon);
  if (!r) r = coord(ps->y, lat);
  if (!r) r = coord(ps->z, depth);
  if (!r && time) {
    cudaError_t e = cudaMemcpyAsync(time, ps->time, n * 8, cudaMemcpyDefault, st);
    if (e) { set_error("copy failed: %s", cudaGetErrorString(e)); r = PG_ERR_CUDA; }
  }
  if (!r && ids) {
    cudaError_t e = cudaMemcpyAsync(ids, ps->id, n * 8, cudaMemcpyDefault, st);
    if (e) { set_error("copy failed: %s", cudaGetErrorString(e)); r = PG_ERR_CUDA; }
  }
  if (!r && steps) {
    cudaError_t e = cudaMemcpyAsync(steps, ps->step, n * 4, cudaMemcpyDefault, st);
    if (e) { set_error("copy failed: %s", cudaGetErrorString(e)); r = PG_ERR_CUDA; }
  }
  if (!r && status) {
    cudaError_t e = cudaMemcpyAsync(status, ps->status, n, cudaMemcpyDefault, st);
    if (e) { set_error("copy failed: %s", cudaGetErrorString(e)); r = PG_ERR_CUDA; }
  }
  cudaError_t e = cudaStreamSynchronize(st);
  if (tmp) dev_free(tmp);
  if (!r && e) { set_error("sync failed: %s", cudaGetErrorString(e)); r = PG_ERR_CUDA; }
  return r;
}

pg_status pg_pset_get_variables(const pg_pset *ps, double *age, double *vars, void *stream) {
  clear_error();
  ARG(ps, "particle set must not be NULL");
  cudaStream_t st = (cudaStream_t)stream;
  const int64_t n = ps->n;
  if (n == 0) return PG_OK;
  if (age) CU(cudaMemcpyAsync(age, ps->age, n * 8, cudaMemcpyDefault, st));
  if (vars)
    for (int j = 0; j < ps->nvar; ++j)
      CU(cudaMemcpyAsync(vars + (size_t)j * n, ps->var + (size_t)j * ps->cap, n * 8,
                         cudaMemcpyDefault, st));
  CU(cudaStreamSynchronize(st));
  return PG_OK;
}

pg_status pg_pset_set_tune(pg_pset *ps, const pg_tune *tune) {
  clear_error();
  ARG(ps && tune, "arguments must not be NULL");
  ARG(tune->block == 0 || (tune->block >= 32 && tune->block <= 1024 && tune->block % 32 == 0),
      "block must be 0 or a multiple of 32 in [32, 1024]");
  ARG(tune->resort_steps >= 0 && tune->chunk_steps >= 0, "negative tuning value");
  ps->tune.block = tune->block ? tune->block : 256;
  ps->tune.resort_steps = tune->resort_steps;
  ps->tune.chunk_steps = tune->chunk_steps ? tune->chunk_steps : 64;
  return PG_OK;
}

pg_status pg_pset_resort(pg_pset *ps, void *stream) {
  clear_error();
  ARG(ps, "particle set must not be NULL");
  int64_t alive = 0;
  CU(launch_resort(ps, (cudaStream_t)stream, &alive));
  CU(cudaStreamSynchronize((cudaStream_t)stream));
  return PG_OK;
}

pg_status pg_pset_moments(const pg_pset *ps, double out[7], void *stream) {
  clear_error();
  ARG(ps && out, "arguments must not be NULL");
  CU(launch_moments(ps, out, (cudaStream_t)stream));
  return PG_OK;
}

// Deliver the output waiting in ring slot k to the caller's hook.
static pg_status deliver_output(pg_pset *ps, int k, pg_output_cb out, pg_record_cb rec,
                                void *user) {
  OutputView hv;
  double t = 0.0;
  CU(ps->out->wait(k, hv, t));
  ps->out->slot[k].pending = false;
  const int64_t n = (int64_t)*hv.count;
  int r;
  if (rec) {
    pg_record R;
    R.time = t; R.n = n; R.nvar = ps->out->nvar; R.var_stride = ps->out->cap;
    R.id = hv.id; R.lon = hv.lon; R.lat = hv.lat; R.depth = hv.depth; R.status = hv.status;
    R.age = hv.age; R.vars = hv.vars;
    r = rec(user, &R);
  } else {
    r = out(user, t, n, hv.id, hv.lon, hv.lat, hv.depth, hv.status);
  }
  if (r != 0) {
    set_error("output callback failed at t = %g", t);
    return PG_ERR_CALLBACK;
  }
  return PG_OK;
}

static pg_status execute_impl(pg_pset *ps, const pg_kernel *k, double runtime, double dt,
                              double output_dt, pg_output_cb out, pg_record_cb rec, int indexed,
                              void *user, void *stream, int64_t *steps_done);
static pg_status execute_loop(pg_pset *ps, const pg_kernel *k, double runtime, double dt,
                              double output_dt, pg_output_cb out, pg_record_cb rec, int indexed,
                              void *user, void *stream, int64_t *steps_done, bool &ran);

// The time range of the alive particles from their device state (after an
// execute that stopped part-way); unchanged when none is alive.
static void refresh_time_range(pg_pset *ps, cudaStream_t st) {
  const int64_t n = ps->n;
  if (n == 0) return;
  std::vector<double> t((size_t)n);
  std::vector<uint8_t> stat((size_t)n);
  if (cudaStreamSynchronize(st) != cudaSuccess ||
      cudaMemcpy(t.data(), ps->time, n * 8, cudaMemcpyDeviceToHost) != cudaSuccess ||
      cudaMemcpy(stat.data(), ps->status, n, cudaMemcpyDeviceToHost) != cudaSuccess) {
    cudaGetLastError();
    return;
  }
  double lo = std::numeric_limits<double>::infinity(), hi = -lo;
  for (int64_t i = 0; i < n; ++i)
    if (stat[i] == 0) { lo = std::min(lo, t[i]); hi = std::max(hi, t[i]); }
  if (lo <= hi) { ps->t_min = lo; ps->t_max = hi; }
}

pg_status pg_execute(pg_pset *ps, const pg_kernel *k, double runtime, double dt,
                     double output_dt, pg_output_cb out, void *user, void *stream,
                     int64_t *steps_done) {
  clear_error();
  return execute_impl(ps, k, runtime, dt, output_dt, out, nullptr, 0, user, stream, steps_done);
}

pg_status pg_execute_records(pg_pset *ps, const pg_kernel *k, double runtime, double dt,
                             double output_dt, int indexed, pg_record_cb rec, void *user,
                             void *stream, int64_t *steps_done) {
  clear_error();
  ARG(indexed == 0 || indexed == 1, "indexed must be 0 or 1");
  return execute_impl(ps, k, runtime, dt, output_dt, nullptr, rec, indexed, user, stream,
                      steps_done);
}

static pg_status execute_impl(pg_pset *ps, const pg_kernel *k, double runtime, double dt,
                              double output_dt, pg_output_cb out, pg_record_cb rec, int indexed,
                              void *user, void *stream, int64_t *steps_done) {
  bool ran = false;
  const pg_status r = execute_loop(ps, k, runtime, dt, output_dt, out, rec, indexed, user, stream,
                                   steps_done, ran);
  if (r && ran) {
    // stopped part-way: the next execute starts from where the particles are
    const std::string msg = pg_last_error();
    refresh_time_range(ps, (cudaStream_t)stream);
    set_error("%s", msg.c_str());
  }
  return r;
}

static pg_status execute_loop(pg_pset *ps, const pg_kernel *k, double runtime, double dt,
                              double output_dt, pg_output_cb out, pg_record_cb rec, int indexed,
                              void *user, void *stream, int64_t *steps_done, bool &ran) {
  ARG(ps && k, "particle set and kernel must not be NULL");
  ARG(std::isfinite(runtime) && runtime >= 0.0, "runtime must be finite and >= 0");
  ARG(std::isfinite(dt) && dt != 0.0, "dt must be finite and non-zero");
  ARG(std::isfinite(output_dt) && output_dt >= 0.0, "output_dt must be finite and >= 0");
  pg_fieldset *fs = ps->fs;
  ARG(fs->nt > 0, "field set has no snapshot times");
  cudaStream_t st = (cudaStream_t)stream;
  if (steps_done) *steps_done = 0;
  if (!fs->streaming) {
    for (int s = 0; s < fs->nt; ++s)
      if (!fs->slabs[s]) {
        set_error("snapshot %d has not been loaded", s);
        return PG_ERR_STATE;
      }
  }
  const double sgn = dt > 0.0 ? 1.0 : -1.0;
  const double t_begin = dt > 0.0 ? ps->t_min : ps->t_max;
  const double t_end = t_begin + sgn * runtime;
  if (fs->nt > 1 && fs->period <= 0.0) {
    const double lo = std::min(dt > 0.0 ? ps->t_min : t_end, t_begin);
    const double hi = std::max(dt > 0.0 ? t_end : ps->t_max, t_begin);
    if (lo < fs->times.front() || hi > fs->times.back()) {
      set_error("execute spans [%g, %g] outside the field times [%g, %g]", lo, hi,
                fs->times.front(), fs->times.back());
      return PG_ERR_TIME;
    }
  }
  if (fs->streaming && fs->nt > 1) {
    double min_gap = std::numeric_limits<double>::infinity();
    for (int s = 0; s + 1 < fs->nt; ++s) min_gap = std::min(min_gap, fs->times[s + 1] - fs->times[s]);
    if (fs->period > 0.0) min_gap = std::min(min_gap, fs->times[0] + fs->period - fs->times.back());
    if (std::fabs(dt) >= min_gap) {
      set_error("streamed fields need |dt| below the snapshot spacing");
      return PG_ERR_UNSUPPORTED;
    }
  }
  StepArgs a;
  {
    pg_status r = resolve_kernel(k, fs, ps->seed, a.k);
    if (r) return r;
  }
  if (k->scheme == PG_RKF45 && a.k.rk_hmax == 0.0) a.k.rk_hmax = std::fabs(dt);
  if (k->scheme == PG_RKF45) a.k.rk_hmin = std::min(a.k.rk_hmin, a.k.rk_hmax);
  const bool ext = (k->beh & (PG_SETTLE | PG_AGE | PG_SAMPLE)) || fs->interp != PG_LINEAR ||
                   k->scheme == PG_RKF45;
  if (ext && ps->pos == PG_POS_CELL) {
    set_error("RKF45, the settle, age and sample behaviours and nearest-neighbour "
              "interpolation need lon/lat/depth positions");
    return PG_ERR_UNSUPPORTED;
  }
  if (ext && ps->pos == PG_POS_F32 && fs->storage != PG_F32) {
    set_error("RKF45, the settle, age and sample behaviours and nearest-neighbour "
              "interpolation need FP32 or FP64 field storage");
    return PG_ERR_UNSUPPORTED;
  }
  if (k->beh & PG_SAMPLE) {
    if (fs->ntr == 0 || ps->nvar != fs->ntr) {
      set_error("the sample behaviour needs scalar fields, added before the particle set");
      return PG_ERR_STATE;
    }
    if (fs->streaming) {
      set_error("scalar fields are sampled from resident snapshots only");
      return PG_ERR_UNSUPPORTED;
    }
    for (size_t q = 0; q < (size_t)fs->ntr * fs->nt; ++q)
      if (!fs->tr_slabs[q]) {
        set_error("snapshot %d of scalar field %d has not been loaded", (int)(q % fs->nt),
                  (int)(q / fs->nt));
        return PG_ERR_STATE;
      }
  }
  a.g = grid_args(fs);
  a.f.nt = fs->nt; a.f.nf = fs->nfields; a.f.times = fs->d_times; a.f.period = fs->period;
  a.f.tab = fs->d_tab;
  a.f.scales = (fs->storage == PG_F16S || fs->storage == PG_BF16S) ? fs->d_scales : nullptr;
  a.f.nearest = fs->interp;
  a.f.ntr = (k->beh & PG_SAMPLE) ? fs->ntr : 0;
  a.f.ttab = fs->d_ttab;
  a.f.tnearest[0] = fs->tr_interp[0]; a.f.tnearest[1] = fs->tr_interp[1];
  a.dt = dt; a.t_end = t_end;
  a.steps_done = ps->d_counter;
  a.err = ps->d_err;
  // everything the time loop allocates is allocated before its first launch,
  // so a failed allocation leaves the particles as they were
  if (ps->tune.resort_steps > 0) CU(prepare_resort(ps));
  const bool want_out = output_dt > 0.0 && (out != nullptr || rec != nullptr);
  if (want_out) {
    if (!ps->out) ps->out = new OutputRing();
    CU(ps->out->prepare(ps->cap, ps->nvar));
  }
  double t_prev_out = t_begin;
  int pending_out = -1;              // ring slot whose output awaits delivery
  CU(cudaMemsetAsync(ps->d_counter, 0, 8, st));
  CU(cudaMemsetAsync(ps->d_err, 0, 4, st));

  const double chunk_len = std::fabs(dt) * (ps->tune.chunk_steps > 0 ? ps->tune.chunk_steps : 64);
  const double resort_len = ps->tune.resort_steps > 0 ? std::fabs(dt) * ps->tune.resort_steps : 0.0;
  double next_out = output_dt > 0.0 ? t_begin + sgn * output_dt : t_end;
  double next_sort = resort_len > 0.0 ? t_begin + sgn * resort_len : t_end;
  int64_t n_active = ps->n;
  // particles arrive in the caller's order (or the order the last execute
  // left): with re-sorting on, the first launch too gets them in Morton
  // order, the deleted ones last (results do not depend on the order)
  if (resort_len > 0.0 && ps->n > 0) CU(launch_resort(ps, st, &n_active));
  double tc = t_begin;
  int guard = 0;
  while (sgn * (t_end - tc) > 0.0) {
    double tn = tc + sgn * chunk_len;
    auto clip = [&](double b) {
      if (sgn * (b - tc) > 0.0 && sgn * (tn - b) > 0.0) tn = b;
    };
    clip(t_end);
    clip(next_out);
    clip(next_sort);
    if (!(sgn * (tn - tc) > 0.0)) {
      set_error("time loop cannot advance from t = %g with dt = %g", tc, dt);
      return PG_ERR_ARG;
    }
    std::vector<int> need;
    if (fs->streaming && fs->nt == 1) {
      need.push_back(0);
      pg_status r = ensure_slots(fs, need, {}, st);
      if (r) return r;
    } else if (fs->streaming) {
      // end the chunk at most B snapshot times after the next one (B = 0: at
      // the next snapshot time); make resident the snapshots bracketing
      // every stage time a step starting in the chunk can reach (B + 3 of
      // them), and start uploading the ones after them into the other
      // slots.  B = (slots - 4) / 2 leaves B + 1 slots for the prefetch,
      // the snapshots the next chunk adds, so a chunk waits for no upload
      // that the previous chunk's compute could have hidden.
      const long long m = snap_counter(fs, tc);
      const long long B = ((long long)fs->slot.size() - 4) / 2;
      if (sgn > 0) {
        clip(snap_time(fs, m + 1 + B));
      } else {
        const double b = snap_time(fs, m - B);
        clip(b < tc ? b : snap_time(fs, m - 1 - B));
      }
      const double adt = std::fabs(dt);
      const double lo_t = sgn > 0 ? tc : std::max(tn - adt, t_end);
      const double hi_t = sgn > 0 ? std::min(tn + adt, t_end) : tc;
      const long long q_lo = snap_counter(fs, lo_t), q_hi = snap_counter(fs, hi_t) + 1;
      for (long long q = q_lo; q <= q_hi; ++q) {
        if (fs->period <= 0.0 && (q < 0 || q >= fs->nt)) continue;
        const int s = snap_of(fs, q);
        if (std::find(need.begin(), need.end(), s) == need.end()) need.push_back(s);
      }
      std::vector<int> pre;
      const long long npre = (long long)fs->slot.size() - (long long)need.size();
      for (long long d = 1; d <= npre; ++d) {
        const long long pq = sgn > 0 ? q_hi + d : q_lo - d;
        if (fs->period <= 0.0 && (pq < 0 || pq >= fs->nt)) break;
        const int s = snap_of(fs, pq);
        if (std::find(need.begin(), need.end(), s) != need.end() ||
            std::find(pre.begin(), pre.end(), s) != pre.end())
          break;
        pre.push_back(s);
      }
      pg_status r = ensure_slots(fs, need, pre, st);
      if (r) return r;
    }
    a.p.n = n_active;
    a.p.x = ps->x; a.p.y = ps->y; a.p.z = ps->z;
    a.p.time = ps->time; a.p.id = ps->id; a.p.step = ps->step; a.p.status = ps->status;
    a.p.age = ps->age; a.p.var = ps->var; a.p.vstride = ps->cap; a.p.hstep = ps->hstep;
    a.t_stop = tn;
    a.t_clip = next_out;
    if (ps->timing) {
      if (ps->ev_used + 2 > ps->ev.size()) {
        for (int q = 0; q < 2; ++q) {
          cudaEvent_t ev;
          CU(cudaEventCreate(&ev));
          ps->ev.push_back(ev);
        }
      }
      CU(cudaEventRecord(ps->ev[ps->ev_used], st));
    }
    a.p.ci = ps->ci; a.p.cj = ps->cj; a.p.ck = ps->ck;
    a.p.fx = ps->fx; a.p.fy = ps->fy; a.p.fz = ps->fz;
    ran = true;
    if (ps->pos == PG_POS_CELL) CU(launch_advect_cell(a, fs->storage, ps->tune.block, st));
    else CU(launch_advect_plain(a, ps->pos, fs->storage, ps->tune.block, st));
    if (ps->timing) {
      CU(cudaEventRecord(ps->ev[ps->ev_used + 1], st));
      ps->ev_used += 2;
    }
    if (fs->streaming) mark_slots_used(fs, need, st);
    tc = tn;
    if (resort_len > 0.0 && tc == next_sort && sgn * (t_end - tc) > 0.0) {
      CU(launch_resort(ps, st, &n_active));
      next_sort = tc + sgn * resort_len;
    }
    if (want_out && (tc == next_out || tc == t_end)) {
      // pack this output and start its copy; then hand the previous one to
      // the caller while the GPU goes on
      CU(ps->out->enqueue(ps, tc, t_prev_out, sgn, indexed, st));
      const int just = ps->out->next ^ 1;
      if (pending_out >= 0) {
        pg_status r = deliver_output(ps, pending_out, out, rec, user);
        if (r) {
          cudaStreamSynchronize(st);
          ps->out->slot[just].pending = false;
          return r;
        }
      }
      pending_out = just;
      t_prev_out = tc;
    }
    if (tc == next_out) next_out = tc + sgn * output_dt;
    if (++guard > 100000000) {
      set_error("time loop made no progress");
      return PG_ERR_STATE;
    }
  }
  if (pending_out >= 0) {
    pg_status r = deliver_output(ps, pending_out, out, rec, user);
    if (r) return r;
  }
  unsigned long long done = 0;
  int err = 0;
  CU(cudaMemcpyAsync(&done, ps->d_counter, 8, cudaMemcpyDeviceToHost, st));
  CU(cudaMemcpyAsync(&err, ps->d_err, 4, cudaMemcpyDeviceToHost, st));
  CU(cudaStreamSynchronize(st));
  if (steps_done) *steps_done = (int64_t)done;
  if (ps->timing) {
    for (size_t q = 0; q + 1 < ps->ev_used; q += 2) {
      float ms = 0.f;
      CU(cudaEventElapsedTime(&ms, ps->ev[q], ps->ev[q + 1]));
      ps->timed_ms += ms;
      ++ps->timed_launches;
    }
    ps->ev_used = 0;
  }
  if (dt > 0.0) { ps->t_min = std::max(ps->t_min, t_end); ps->t_max = std::max(ps->t_max, t_end); }
  else { ps->t_min = std::min(ps->t_min, t_end); ps->t_max = std::min(ps->t_max, t_end); }
  if (err) {
    set_error("a kernel recorded internal error %d", err);
    return PG_ERR_DEVICE;
  }
  return PG_OK;
}

pg_status pg_pset_kernel_timing(pg_pset *ps, int enable, double *total_ms, int64_t *launches) {
  clear_error();
  ARG(ps, "particle set must not be NULL");
  if (total_ms) *total_ms = ps->timed_ms;
  if (launches) *launches = ps->timed_launches;
  if (enable >= 0) {
    ps->timing = enable != 0;
    ps->timed_ms = 0.0;
    ps->timed_launches = 0;
    ps->ev_used = 0;
  }
  return PG_OK;
}

pg_status pg_launch_count(int64_t *count) {
  clear_error();
  ARG(count, "count must not be NULL");
  *count = (int64_t)g_launches.load();
  return PG_OK;
}

pg_status pg_pset_save(const pg_pset *ps, const char *path) {
  clear_error();
  ARG(ps && path, "arguments must not be NULL");
  const int64_t n = ps->n;
  // raw array bytes keep FP32 and cell-form state bit for bit
  const auto arrays = state_arrays(arrays_of(ps), ps->pos, ps->nvar, ps->cap);
  std::vector<std::vector<char>> host(arrays.size());
  for (size_t q = 0; q < arrays.size(); ++q) {
    host[q].resize((size_t)n * arrays[q].second);
    if (n) CU(cudaMemcpy(host[q].data(), arrays[q].first, host[q].size(), cudaMemcpyDeviceToHost));
  }
  FILE *f = fopen(path, "wb");
  if (!f) {
    set_error("cannot open %s for writing", path);
    return PG_ERR_ARG;
  }
  const char magic[8] = {'P', 'G', 'P', 'S', 'E', 'T', '0', '3'};
  const int32_t pos = ps->pos, nvar = ps->nvar;
  bool ok = fwrite(magic, 8, 1, f) == 1 && fwrite(&pos, 4, 1, f) == 1 &&
            fwrite(&nvar, 4, 1, f) == 1 &&
            fwrite(&n, 8, 1, f) == 1 && fwrite(&ps->seed, 8, 1, f) == 1 &&
            fwrite(&ps->t_min, 8, 1, f) == 1 && fwrite(&ps->t_max, 8, 1, f) == 1;
  for (size_t q = 0; ok && q < host.size(); ++q)
    if (n) ok = fwrite(host[q].data(), 1, host[q].size(), f) == host[q].size();
  if (fclose(f) != 0) ok = false;
  if (!ok) {
    set_error("write to %s failed", path);
    return PG_ERR_ARG;
  }
  return PG_OK;
}

pg_status pg_pset_restore(pg_fieldset *fs, const char *path, pg_pset **out) {
  clear_error();
  ARG(fs && path && out, "arguments must not be NULL");
  FILE *f = fopen(path, "rb");
  if (!f) {
    set_error("cannot open %s", path);
    return PG_ERR_ARG;
  }
  char magic[8];
  int32_t pos = 0, nvar = 0;
  int64_t n = 0;
  uint64_t seed = 0;
  double tmin = 0, tmax = 0;
  bool ok = fread(magic, 8, 1, f) == 1 && memcmp(magic, "PGPSET03", 8) == 0 &&
            fread(&pos, 4, 1, f) == 1 && fread(&nvar, 4, 1, f) == 1 && nvar >= 0 && nvar <= 2 &&
            fread(&n, 8, 1, f) == 1 && fread(&seed, 8, 1, f) == 1 &&
            fread(&tmin, 8, 1, f) == 1 && fread(&tmax, 8, 1, f) == 1 &&
            (pos == PG_POS_F64 || pos == PG_POS_F32 || pos == PG_POS_CELL) && n >= 0 &&
            n < ((int64_t)1 << 40);
  std::vector<std::vector<char>> host;
  if (ok) {
    const auto sizes = state_arrays(PsetArrays(), pos, nvar, n);
    host.resize(sizes.size());
    for (size_t q = 0; ok && q < sizes.size(); ++q) {
      host[q].resize((size_t)n * sizes[q].second);
      if (n) ok = fread(host[q].data(), 1, host[q].size(), f) == host[q].size();
    }
  }
  fclose(f);
  if (!ok) {
    set_error("%s is not a particle-set checkpoint", path);
    return PG_ERR_ARG;
  }
  if (nvar != fs->ntr) {
    set_error("checkpoint %s has %d sampled variables, the field set %d scalar fields", path,
              (int)nvar, fs->ntr);
    return PG_ERR_ARG;
  }
  // create an empty set of the right form, then fill it raw
  pg_pset *ps = nullptr;
  pg_status r = pg_pset_create(fs, 0, nullptr, nullptr, nullptr, nullptr, tmin, nullptr, 0, pos,
                               seed, &ps);
  if (r) return r;
  if (n) {
    PsetArrays B;
    r = alloc_arrays(B, pos, n, nvar);
    if (r) { pg_pset_destroy(ps); return r; }
    const auto arrays = state_arrays(B, pos, nvar, n);
    cudaError_t e = cudaSuccess;
    for (size_t q = 0; e == cudaSuccess && q < arrays.size(); ++q)
      e = cudaMemcpy(arrays[q].first, host[q].data(), host[q].size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
      B.free_all();
      pg_pset_destroy(ps);
      set_error("restore copy failed: %s", cudaGetErrorString(e));
      return PG_ERR_CUDA;
    }
    arrays_of(ps).free_all();
    set_arrays(ps, B);
    ps->cap = n;
  }
  ps->n = n;
  ps->t_min = tmin; ps->t_max = tmax;
  *out = ps;
  return PG_OK;
}

pg_status pg_pset_destroy(pg_pset *ps) {
  clear_error();
  if (!ps) return PG_OK;
  cudaDeviceSynchronize();
  arrays_of(ps).free_all();
  ps->alt.free_all();
  dev_free(ps->d_counter);
  dev_free(ps->d_err);
  dev_free(ps->sort_scratch);
  dev_free(ps->diag_scratch);
  for (cudaEvent_t ev : ps->ev) cudaEventDestroy(ev);
  delete ps->out;
  delete ps;
  return PG_OK;
}

}  // extern "C"
