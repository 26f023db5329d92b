// surrogate.cu -- the learned 24-hour flow map: features, displacement,
// and the run loop in which RK4 (Sect. 2.1.1) checks the network and takes
// over for the particles it rejects.  The features and the displacement are
// those of surrogate_features.cuh.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <vector>

#include "surrogate_features.cuh"
#include "pg_host.h"

namespace pg {

namespace {

constexpr int kFeat = kSurFeat;

__device__ __forceinline__ int find_cell(const float *x, int n, float p) {
  int lo = 0, hi = n - 1;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (x[mid] <= p) lo = mid; else hi = mid;
  }
  return lo;
}

__global__ void features_kernel(GridArgs g, FieldArgs f, const float *lon, const float *lat,
                                const float *dep, const double *time, const uint8_t *status,
                                int64_t n, float *out, int *err) {
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n;
       p += (int64_t)gridDim.x * blockDim.x) {
    float *o = out + p * kFeat;
    float v[kFeat];
    if (status[p] != 0) {
#pragma unroll
      for (int q = 0; q < kFeat; ++q) o[q] = 0.f;
      continue;
    }
    const int r = surrogate_features(g, f, lon[p], lat[p], dep[p], time[p], v);
    if (r) {
      atomicCAS(err, 0, r);
      continue;
    }
#pragma unroll
    for (int q = 0; q < kFeat; ++q) o[q] = v[q];
  }
}

// Apply predicted displacements over `horizon` seconds.
__global__ void apply_kernel(GridArgs g, float *lon, float *lat, float *dep, double *time,
                             uint32_t *step, uint8_t *status, int64_t n, const float *y,
                             double horizon) {
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n;
       p += (int64_t)gridDim.x * blockDim.x) {
    if (status[p] != 0) continue;
    float l = lon[p], a = lat[p], d = dep[p];
    const uint8_t st = surrogate_apply(g, l, a, d, y[p * 3 + 0], y[p * 3 + 1], y[p * 3 + 2]);
    if (st) { status[p] = st; continue; }
    lon[p] = l; lat[p] = a; dep[p] = d;
    time[p] += horizon;
    step[p] += 1;
  }
}

// Displacement between two states of the same particles (same order):
// cells of lon (shortest way round) and lat, 100 m units of depth.
__global__ void displacement_kernel(GridArgs g, const float *lon0, const float *lat0,
                                    const float *dep0, const float *lon1, const float *lat1,
                                    const float *dep1, int64_t n, float *y) {
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n;
       p += (int64_t)gridDim.x * blockDim.x) {
    float dl = lon1[p] - lon0[p];
    if (g.periodic) {
      if (dl > 180.f) dl -= 360.f;
      if (dl < -180.f) dl += 360.f;
    }
    y[p * 3 + 0] = dl / g.df[0];
    y[p * 3 + 1] = (lat1[p] - lat0[p]) / g.df[1];
    y[p * 3 + 2] = (dep1[p] - dep0[p]) / kSurDepthUnit;
  }
}

// Position error (in cells; depth in units of the local layer) between the
// network's state and RK4's; rejects particles above the threshold, and any
// particle alive at the block's start that the network or the checking RK4 deleted
// within the block (RK4 from the block's start then decides).  err_sum[0] +=
// error over particles both keep alive, err_sum[1] += count.
__global__ void check_kernel(GridArgs g, const float *lon_a, const float *lat_a,
                             const float *dep_a, const uint8_t *st_a, const float *lon_b,
                             const float *lat_b, const float *dep_b, const uint8_t *st_b,
                             const uint8_t *st_ckpt, int64_t n, float threshold, uint8_t *reject,
                             double *err_sum, unsigned long long *n_reject) {
  double e_acc = 0.0, c_acc = 0.0;
  unsigned long long r_acc = 0;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n;
       p += (int64_t)gridDim.x * blockDim.x) {
    uint8_t rj = 0;
    if (st_ckpt[p] != 0) {
      rj = 0;              // deleted before the block: stays deleted
    } else if (st_a[p] != 0 || st_b[p] != 0) {
      rj = 1;              // a deletion inside the block is decided by RK4 alone
    } else {
      float dl = lon_a[p] - lon_b[p];
      if (g.periodic) {
        if (dl > 180.f) dl -= 360.f;
        if (dl < -180.f) dl += 360.f;
      }
      float e = fmaxf(fabsf(dl) / g.df[0], fabsf(lat_a[p] - lat_b[p]) / g.df[1]);
      if (g.nz > 1) {
        const int k = find_cell(g.depthf, g.nz, fminf(fmaxf(dep_b[p], g.depthf[0]), g.depthf[g.nz - 1]));
        e = fmaxf(e, fabsf(dep_a[p] - dep_b[p]) / (g.depthf[k + 1] - g.depthf[k]));
      }
      if (!(e <= threshold)) rj = 1;
      e_acc += (double)fminf(e, 1e6f);
      c_acc += 1.0;
    }
    reject[p] = rj;
    r_acc += rj;
  }
  atomicAdd(&err_sum[0], e_acc);
  atomicAdd(&err_sum[1], c_acc);
  atomicAdd(n_reject, r_acc);
}

// The rejected particles are re-integrated as a dense set: their
// checkpoint states are packed, in particle order, into the arrays of a
// second set (position k of the rejected ones given by an exclusive scan of
// the reject flags), advanced there, and written back to their places.
__global__ void flags_kernel(const uint8_t *reject, int64_t n, uint32_t *flags) {
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n;
       p += (int64_t)gridDim.x * blockDim.x)
    flags[p] = reject[p] ? 1u : 0u;
}

struct SetPtrs {
  float *x, *y, *z;
  double *time;
  uint64_t *id;
  uint32_t *step;
  uint8_t *status;
};

// Particles p0 .. p0 + n - 1; offs is the exclusive scan of their flags and
// base the number of rejected particles before p0.
__global__ void pack_rejected_kernel(const uint8_t *reject, const uint32_t *offs, int64_t p0,
                                     int64_t n, uint32_t base, SetPtrs src, SetPtrs dst,
                                     uint32_t *idx) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t p = p0 + i;
    if (!reject[p]) continue;
    const uint32_t k = base + offs[i];
    idx[k] = (uint32_t)p;
    dst.x[k] = src.x[p]; dst.y[k] = src.y[p]; dst.z[k] = src.z[p];
    dst.time[k] = src.time[p]; dst.id[k] = src.id[p]; dst.step[k] = src.step[p];
    dst.status[k] = src.status[p];
  }
}

__global__ void unpack_rejected_kernel(const uint32_t *idx, int64_t m, SetPtrs src, SetPtrs dst) {
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < m;
       k += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t p = idx[k];
    dst.x[p] = src.x[k]; dst.y[p] = src.y[k]; dst.z[p] = src.z[k];
    dst.time[p] = src.time[k]; dst.step[p] = src.step[k]; dst.status[p] = src.status[k];
  }
}

SetPtrs set_ptrs(pg_pset *ps) {
  return SetPtrs{(float *)ps->x, (float *)ps->y, (float *)ps->z, ps->time, ps->id, ps->step,
                 ps->status};
}

int grid_of(int64_t n, int sm) {
  int64_t g = (n + 255) / 256;
  if (g > (int64_t)sm * 16) g = (int64_t)sm * 16;
  return (int)(g < 1 ? 1 : g);
}

FieldArgs field_args(const pg_fieldset *fs) {
  FieldArgs f;
  f.nt = fs->nt; f.nf = fs->nfields; f.times = fs->d_times; f.period = fs->period;
  f.tab = fs->d_tab;
  f.scales = nullptr;
  return f;
}

}  // namespace

cudaError_t launch_resort(pg_pset *ps, cudaStream_t st, int64_t *n_alive);
int64_t scan_max_entries();
size_t scan_scratch_words(int64_t m);
cudaError_t exclusive_scan_u32(const uint32_t *in, uint32_t *out, int64_t m, uint32_t *tmp,
                               cudaStream_t st);

}  // namespace pg

using namespace pg;

#define CUS(call)                                                                     \
  do {                                                                                \
    cudaError_t e_ = (call);                                                          \
    if (e_ != cudaSuccess) {                                                          \
      set_error("%s failed: %s", #call, cudaGetErrorString(e_));                      \
      return e_ == cudaErrorMemoryAllocation ? PG_ERR_NOMEM : PG_ERR_CUDA;            \
    }                                                                                 \
  } while (0)

static pg_status check_pset(const pg_pset *ps) {
  if (!ps) {
    set_error("invalid argument: null particle set");
    return PG_ERR_ARG;
  }
  if (ps->pos != PG_POS_F32 || ps->fs->storage != PG_F32 || ps->fs->streaming) {
    set_error("the surrogate needs FP32 positions on a resident FP32 field set");
    return PG_ERR_UNSUPPORTED;
  }
  return PG_OK;
}

extern "C" {

pg_status pg_surrogate_features(const pg_pset *ps, float *x, void *stream) {
  clear_error();
  pg_status r = check_pset(ps);
  if (r) return r;
  if (!x && ps->n) { set_error("invalid argument: null output"); return PG_ERR_ARG; }
  cudaStream_t st = (cudaStream_t)stream;
  if (ps->n == 0) return PG_OK;
  CUS(cudaMemsetAsync(ps->d_err, 0, 4, st));
  features_kernel<<<grid_of(ps->n, ps->fs->sm_count), 256, 0, st>>>(
      grid_args_of(ps->fs), field_args(ps->fs), (const float *)ps->x, (const float *)ps->y,
      (const float *)ps->z, ps->time, ps->status, ps->n, x, ps->d_err);
  note_launches(1);
  CUS(cudaGetLastError());
  int err = 0;
  CUS(cudaMemcpyAsync(&err, ps->d_err, 4, cudaMemcpyDeviceToHost, st));
  CUS(cudaStreamSynchronize(st));
  if (err) { set_error("feature kernel recorded internal error %d", err); return PG_ERR_DEVICE; }
  return PG_OK;
}

pg_status pg_surrogate_apply(pg_pset *ps, const float *y, double horizon, void *stream) {
  clear_error();
  pg_status r = check_pset(ps);
  if (r) return r;
  if ((!y && ps->n) || !std::isfinite(horizon)) { set_error("invalid argument"); return PG_ERR_ARG; }
  cudaStream_t st = (cudaStream_t)stream;
  if (ps->n) {
    apply_kernel<<<grid_of(ps->n, ps->fs->sm_count), 256, 0, st>>>(
        grid_args_of(ps->fs), (float *)ps->x, (float *)ps->y, (float *)ps->z, ps->time, ps->step,
        ps->status, ps->n, y, horizon);
    note_launches(1);
    CUS(cudaGetLastError());
  }
  ps->t_min += horizon;
  ps->t_max += horizon;
  return PG_OK;
}

pg_status pg_pset_displacement(const pg_pset *a, const pg_pset *b, float *y, void *stream) {
  clear_error();
  pg_status r = check_pset(a);
  if (!r) r = check_pset(b);
  if (r) return r;
  if (a->n != b->n || a->fs != b->fs || (!y && a->n)) {
    set_error("invalid argument: sets of equal size on one field set and an output");
    return PG_ERR_ARG;
  }
  if (a->n == 0) return PG_OK;
  cudaStream_t st = (cudaStream_t)stream;
  displacement_kernel<<<grid_of(a->n, a->fs->sm_count), 256, 0, st>>>(
      grid_args_of(a->fs), (const float *)a->x, (const float *)a->y, (const float *)a->z,
      (const float *)b->x, (const float *)b->y, (const float *)b->z, a->n, y);
  note_launches(1);
  CUS(cudaGetLastError());
  return PG_OK;
}

pg_status pg_mlp_forward(pg_mlp *net, const float *x, int64_t M, float *y, void *stream);

// The surrogate run: blocks of `check_every` network steps of `horizon`
// seconds.  The last step of every block is judged by RK4 (dt_check) from
// the same state; particles whose error exceeds `threshold` cells (or whose
// status differs) are re-integrated with RK4 from the block's start, the
// others take RK4's state for that step.
pg_status pg_surrogate_run(pg_pset *ps, pg_mlp *net, const pg_kernel *k, int nsteps,
                           int check_every, double horizon, double dt_check, double threshold,
                           pg_surrogate_stats *stats, void *stream) {
  clear_error();
  pg_status r = check_pset(ps);
  if (r) return r;
  if (!net || !k || nsteps < 1 || check_every < 1 || !(horizon > 0.0) || !(dt_check > 0.0) ||
      !(threshold >= 0.0)) {
    set_error("invalid argument: need a network, a kernel, nsteps, check_every >= 1, horizon, "
              "dt_check > 0 and threshold >= 0");
    return PG_ERR_ARG;
  }
  cudaStream_t st = (cudaStream_t)stream;
  const int64_t n = ps->n;
  const int sm = ps->fs->sm_count;
  pg_surrogate_stats S{};
  // buffers: features, outputs, reject flags, checkpoint and check sets
  float *x = nullptr, *y = nullptr;
  uint8_t *rej = nullptr;
  double *esum = nullptr;
  unsigned long long *nrej = nullptr;
  uint32_t *flags = nullptr, *offs = nullptr, *scan_tmp = nullptr, *idx = nullptr;
  pg_pset *ckpt = nullptr, *chk = nullptr, *rset = nullptr;
  cudaEvent_t e0, e1, e2;
  CUS(cudaEventCreate(&e0));
  CUS(cudaEventCreate(&e1));
  CUS(cudaEventCreate(&e2));
  auto cleanup = [&]() {
    dev_free(x); dev_free(y); dev_free(rej); dev_free(esum); dev_free(nrej);
    dev_free(flags); dev_free(offs); dev_free(scan_tmp); dev_free(idx);
    if (ckpt) pg_pset_destroy(ckpt);
    if (chk) pg_pset_destroy(chk);
    if (rset) pg_pset_destroy(rset);
    cudaEventDestroy(e0); cudaEventDestroy(e1); cudaEventDestroy(e2);
  };
  cudaError_t e = dev_alloc((void **)&x, (size_t)std::max<int64_t>(n, 1) * kFeat * 4);
  if (e == cudaSuccess) e = dev_alloc((void **)&y, (size_t)std::max<int64_t>(n, 1) * 3 * 4);
  if (e == cudaSuccess) e = dev_alloc((void **)&rej, (size_t)std::max<int64_t>(n, 1));
  if (e == cudaSuccess) e = dev_alloc((void **)&esum, 16);
  if (e == cudaSuccess) e = dev_alloc((void **)&nrej, 8);
  // compaction of the rejected particles, in pieces of at most one scan
  const int64_t piece = std::min<int64_t>(std::max<int64_t>(n, 1), scan_max_entries());
  if (e == cudaSuccess) e = dev_alloc((void **)&flags, (size_t)piece * 4);
  if (e == cudaSuccess) e = dev_alloc((void **)&offs, (size_t)piece * 4);
  if (e == cudaSuccess) e = dev_alloc((void **)&scan_tmp, scan_scratch_words(piece) * 4);
  if (e == cudaSuccess) e = dev_alloc((void **)&idx, (size_t)std::max<int64_t>(n, 1) * 4);
  if (e != cudaSuccess) {
    cleanup();
    set_error("surrogate buffers: %s", cudaGetErrorString(e));
    return PG_ERR_NOMEM;
  }
  // two more sets with the same arrays' shapes
  std::vector<double> zeros(1, 0.0);
  if ((r = pg_pset_create(ps->fs, 0, nullptr, nullptr, nullptr, nullptr, 0.0, nullptr, 0,
                          PG_POS_F32, ps->seed, &ckpt)) ||
      (r = pg_pset_create(ps->fs, 0, nullptr, nullptr, nullptr, nullptr, 0.0, nullptr, 0,
                          PG_POS_F32, ps->seed, &chk)) ||
      (r = pg_pset_create(ps->fs, 0, nullptr, nullptr, nullptr, nullptr, 0.0, nullptr, 0,
                          PG_POS_F32, ps->seed, &rset))) {
    cleanup();
    return r;
  }
  auto copy_set = [&](pg_pset *dst, const pg_pset *src) -> cudaError_t {
    if (dst->cap < src->n) {
      PsetArrays A;
      if (alloc_arrays(A, PG_POS_F32, src->n, dst->nvar) != PG_OK)
        return cudaErrorMemoryAllocation;
      pset_arrays(dst).free_all();
      pset_set_arrays(dst, A);
      dst->cap = src->n;
    }
    const size_t m = (size_t)src->n;
    cudaError_t q = cudaMemcpyAsync(dst->x, src->x, m * 4, cudaMemcpyDeviceToDevice, st);
    if (!q) q = cudaMemcpyAsync(dst->y, src->y, m * 4, cudaMemcpyDeviceToDevice, st);
    if (!q) q = cudaMemcpyAsync(dst->z, src->z, m * 4, cudaMemcpyDeviceToDevice, st);
    if (!q) q = cudaMemcpyAsync(dst->time, src->time, m * 8, cudaMemcpyDeviceToDevice, st);
    if (!q) q = cudaMemcpyAsync(dst->id, src->id, m * 8, cudaMemcpyDeviceToDevice, st);
    if (!q) q = cudaMemcpyAsync(dst->step, src->step, m * 4, cudaMemcpyDeviceToDevice, st);
    if (!q) q = cudaMemcpyAsync(dst->status, src->status, m, cudaMemcpyDeviceToDevice, st);
    dst->n = src->n;
    dst->t_min = src->t_min;
    dst->t_max = src->t_max;
    return q;
  };
  // a network step: features, network, displacement -- one fused tcgen05
  // kernel for the surrogate's network shape, else three kernels
  const bool fused_step = mlp_fused_step_ok(net);
  auto network_step = [&]() -> pg_status {
    if (fused_step) {
      SurrogateStepIO io;
      io.g = grid_args_of(ps->fs);
      io.f = field_args(ps->fs);
      io.lon = (float *)ps->x; io.lat = (float *)ps->y; io.dep = (float *)ps->z;
      io.time = ps->time; io.step = ps->step; io.status = ps->status;
      io.n = ps->n; io.horizon = horizon; io.ferr = ps->d_err;
      const pg_status q = mlp_fused_step(net, io, st);
      if (!q) { ps->t_min += horizon; ps->t_max += horizon; }
      return q;
    }
    pg_status q = pg_surrogate_features(ps, x, st);
    if (!q) q = pg_mlp_forward(net, x, n, y, st);
    if (!q) q = pg_surrogate_apply(ps, y, horizon, st);
    return q;
  };
  pg_tune keep_order{ps->tune.block > 0 ? ps->tune.block : 256, 0, 64};
  float ms_net = 0.f, ms_rk = 0.f;
  const auto t_start = std::chrono::steady_clock::now();
  int done_steps = 0;
  while (done_steps < nsteps && r == PG_OK) {
    const int blk = std::min(check_every, nsteps - done_steps);
    // Morton order at the start of every block (when the set's tuning asks
    // for re-sorts), for the locality of the features, checks and fallback
    if (ps->tune.resort_steps > 0 && n > 0) {
      int64_t alive = 0;
      e = launch_resort(ps, st, &alive);
      if (e) { r = PG_ERR_CUDA; set_error("re-sort: %s", cudaGetErrorString(e)); break; }
    }
    e = copy_set(ckpt, ps);
    if (e) { r = PG_ERR_CUDA; set_error("checkpoint copy: %s", cudaGetErrorString(e)); break; }
    cudaEventRecord(e0, st);
    for (int s = 0; s < blk - 1 && r == PG_OK; ++s) r = network_step();
    if (r) break;
    // judge the last step of the block: RK4 on a copy, the network on ps
    e = copy_set(chk, ps);
    if (e) { r = PG_ERR_CUDA; set_error("check copy: %s", cudaGetErrorString(e)); break; }
    if ((r = network_step())) break;
    cudaEventRecord(e1, st);
    chk->tune = keep_order;
    int64_t rk = 0;
    if ((r = pg_execute(chk, k, horizon, dt_check, 0.0, nullptr, nullptr, st, &rk))) break;
    S.rk4_particle_steps += rk;
    CUS(cudaMemsetAsync(esum, 0, 16, st));
    CUS(cudaMemsetAsync(nrej, 0, 8, st));
    check_kernel<<<grid_of(n, sm), 256, 0, st>>>(
        grid_args_of(ps->fs), (const float *)ps->x, (const float *)ps->y, (const float *)ps->z,
        ps->status, (const float *)chk->x, (const float *)chk->y, (const float *)chk->z,
        chk->status, ckpt->status, n, (float)threshold, rej, esum, nrej);
    note_launches(1);
    double h_esum[2];
    unsigned long long h_nrej = 0;
    CUS(cudaMemcpyAsync(h_esum, esum, 16, cudaMemcpyDeviceToHost, st));
    CUS(cudaMemcpyAsync(&h_nrej, nrej, 8, cudaMemcpyDeviceToHost, st));
    CUS(cudaStreamSynchronize(st));
    S.checked += (int64_t)h_esum[1];
    S.error_sum += h_esum[0];
    S.rejected += (int64_t)h_nrej;
    // everyone takes RK4's state for the checked step ...
    if ((e = copy_set(ps, chk))) { r = PG_ERR_CUDA; set_error("%s", cudaGetErrorString(e)); break; }
    // ... and the rejected re-integrate the whole block from the checkpoint,
    // packed into a dense set
    if (h_nrej > 0) {
      const int64_t m = (int64_t)h_nrej;
      if (rset->cap < m) {
        PsetArrays A;
        if (alloc_arrays(A, PG_POS_F32, m, rset->nvar) != PG_OK) {
          r = PG_ERR_NOMEM;
          set_error("surrogate fallback set of %lld particles", (long long)m);
          break;
        }
        pset_arrays(rset).free_all();
        pset_set_arrays(rset, A);
        rset->cap = m;
      }
      const SetPtrs cp = set_ptrs(ckpt), rp = set_ptrs(rset), pp = set_ptrs(ps);
      uint32_t base = 0;
      for (int64_t p0 = 0; p0 < n && !e; p0 += piece) {
        const int64_t len = std::min(piece, n - p0);
        const int g = grid_of(len, sm);
        flags_kernel<<<g, 256, 0, st>>>(rej + p0, len, flags);
        e = exclusive_scan_u32(flags, offs, len, scan_tmp, st);
        if (e) break;
        pack_rejected_kernel<<<g, 256, 0, st>>>(rej, offs, p0, len, base, cp, rp, idx);
        note_launches(2);
        if (p0 + len < n) {
          // the next piece's rejected particles follow this piece's
          uint32_t last_off = 0, last_flag = 0;
          e = cudaMemcpyAsync(&last_off, offs + len - 1, 4, cudaMemcpyDeviceToHost, st);
          if (!e) e = cudaMemcpyAsync(&last_flag, flags + len - 1, 4, cudaMemcpyDeviceToHost, st);
          if (!e) e = cudaStreamSynchronize(st);
          base += last_off + last_flag;
        }
      }
      if (e) { r = PG_ERR_CUDA; set_error("fallback packing: %s", cudaGetErrorString(e)); break; }
      rset->n = m;
      rset->t_min = ckpt->t_min;
      rset->t_max = ckpt->t_max;
      rset->tune = keep_order;
      if ((r = pg_execute(rset, k, blk * horizon, dt_check, 0.0, nullptr, nullptr, st, &rk))) break;
      unpack_rejected_kernel<<<grid_of(m, sm), 256, 0, st>>>(idx, m, rp, pp);
      note_launches(1);
      S.rk4_particle_steps += rk;
    }
    cudaEventRecord(e2, st);
    CUS(cudaEventSynchronize(e2));
    float a = 0.f, b = 0.f;
    cudaEventElapsedTime(&a, e0, e1);
    cudaEventElapsedTime(&b, e1, e2);
    ms_net += a;
    ms_rk += b;
    S.network_steps += (int64_t)(blk - 1) * n + n;
    done_steps += blk;
  }
  S.seconds_network = ms_net * 1e-3;
  S.seconds_rk4 = ms_rk * 1e-3;
  S.seconds_total =
      std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count();
  if (stats) *stats = S;
  cleanup();
  return r;
}

}  // extern "C"
