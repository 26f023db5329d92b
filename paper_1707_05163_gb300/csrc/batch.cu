// batch.cu -- many releases in one persistent launch per window, the window
// loop captured in a CUDA graph, and an autotuner for block size and re-sort
// interval.
//
// Each release is a particle set (the repeated releases of Sect. 3) with its
// own kernel, dt and runtime; all share one field set.  A window (one day by
// default) of simulated time is one launch of the persistent kernel, which
// walks a work list of (release, tile) pairs ordered heaviest first (most
// steps per window) with one atomic per tile, so releases of very different
// cost balance across the SMs.  With re-sorting on, large releases are
// sorted before the first window and every k windows, in fixed-pointer mode
// so the sequence of launches is the same on every replay and can be captured
// once.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <fstream>
#include <sstream>
#include <string>

#include "advect_plain.cuh"
#include "pg_host.h"

namespace pg {

cudaError_t prepare_resort(pg_pset *ps);
cudaError_t launch_resort(pg_pset *ps, cudaStream_t st, int64_t *n_alive);

namespace {

// The batch kernel for one field shape and geometry: launch it (bps null) or
// report its occupancy in blocks per SM.
template <typename Store, int GEO>
cudaError_t batch_geo(const BatchArgs &b, int block, int grid, cudaStream_t st, int *bps) {
  auto kern = b.f.nf == 3 ? advect_batch_kernel<Store, 3, true, GEO>
            : (b.g.nz > 1 ? advect_batch_kernel<Store, 2, true, GEO>
                          : advect_batch_kernel<Store, 2, false, GEO>);
  if (bps) return cudaOccupancyMaxActiveBlocksPerMultiprocessor(bps, kern, block, 0);
  kern<<<grid, block, 0, st>>>(b);
  note_launches(1);
  return cudaGetLastError();
}

template <typename Store>
cudaError_t batch_store(const BatchArgs &b, int block, int grid, cudaStream_t st, int *bps) {
  switch (geo_of(b.g)) {
    case GEO_FLAT: return batch_geo<Store, GEO_FLAT>(b, block, grid, st, bps);
    case GEO_SPH: return batch_geo<Store, GEO_SPH>(b, block, grid, st, bps);
    default: return batch_geo<Store, GEO_SPH_PER>(b, block, grid, st, bps);
  }
}

cudaError_t batch_op(const BatchArgs &b, int storage, int block, int grid, cudaStream_t st,
                     int *bps) {
  switch (storage) {
    case PG_F32: return batch_store<float>(b, block, grid, st, bps);
    case PG_F16S: return batch_store<__half>(b, block, grid, st, bps);
    case PG_BF16S: return batch_store<__nv_bfloat16>(b, block, grid, st, bps);
    default: return cudaErrorInvalidValue;
  }
}

// Releases at least this large are re-sorted; smaller ones stay in L2.
constexpr int64_t kResortMin = 65536;

struct Batch {
  pg_fieldset *fs = nullptr;
  std::vector<pg_pset *> ps;
  std::vector<BatchRelease> rel;
  BatchRelease *d_rel = nullptr;
  int2 *d_tiles = nullptr;
  int ntiles = 0;
  int *d_next = nullptr;      // one work-list cursor per window
  int nwin = 0;
  double t_begin = 0.0, window = 0.0;
  unsigned long long *d_steps = nullptr;
  int *d_err = nullptr;
  ~Batch() {
    dev_free(d_rel); dev_free(d_tiles); dev_free(d_next); dev_free(d_steps); dev_free(d_err);
  }
};

// Morton sort of every release large enough to gain from it.
cudaError_t sort_releases(Batch &B, cudaStream_t st) {
  cudaError_t e = cudaSuccess;
  for (pg_pset *p : B.ps)
    if (p->n >= kResortMin && (e = launch_resort(p, st, nullptr)) != cudaSuccess) return e;
  return e;
}

// Enqueue windows [w0, w1) with the given block size and re-sort interval
// (first_sort: with re-sorting on, sort before window 0 as well).
cudaError_t enqueue_windows(Batch &B, int w0, int w1, int block, int resort_every,
                            cudaStream_t st, bool first_sort = true) {
  const pg_fieldset *fs = B.fs;
  BatchArgs b;
  b.g = grid_args_of(fs);
  b.f.nt = fs->nt; b.f.nf = fs->nfields; b.f.times = fs->d_times; b.f.period = fs->period;
  b.f.tab = fs->d_tab;
  b.f.scales = (fs->storage == PG_F16S || fs->storage == PG_BF16S) ? fs->d_scales : nullptr;
  b.rel = B.d_rel;
  b.tiles = B.d_tiles;
  b.ntiles = B.ntiles;
  b.steps_done = B.d_steps;
  b.err = B.d_err;
  int bps = 0;
  cudaError_t e = batch_op(b, fs->storage, block, 0, st, &bps);
  if (e != cudaSuccess) return e;
  const int grid = std::max(1, std::min(bps * fs->sm_count, B.ntiles));
  // with re-sorting on, the first window too runs on Morton-ordered particles
  if (first_sort && resort_every > 0 && w0 == 0 && w1 > 0) {
    if ((e = sort_releases(B, st)) != cudaSuccess) return e;
  }
  for (int w = w0; w < w1; ++w) {
    b.next_tile = B.d_next + w;
    b.t_stop = B.t_begin + (double)(w + 1) * B.window;
    if ((e = batch_op(b, fs->storage, block, grid, st, nullptr)) != cudaSuccess) return e;
    if (resort_every > 0 && (w + 1) % resort_every == 0 && w + 1 < B.nwin) {
      for (pg_pset *p : B.ps)
        if (p->n >= kResortMin && (e = launch_resort(p, st, nullptr)) != cudaSuccess) return e;
    }
  }
  return cudaSuccess;
}

struct Backup {
  std::vector<std::vector<std::pair<void *, size_t>>> bufs;   // per release: (copy, bytes)
  ~Backup() {
    for (auto &v : bufs)
      for (auto &q : v) dev_free(q.first);
  }
};

std::vector<std::pair<void *, size_t>> live_arrays(pg_pset *p) {
  const size_t n = (size_t)p->n;
  return {{p->x, n * 4}, {p->y, n * 4}, {p->z, n * 4}, {p->time, n * 8},
          {p->id, n * 8}, {p->step, n * 4}, {p->status, n}};
}

cudaError_t save_state(Batch &B, Backup &bk, cudaStream_t st) {
  bk.bufs.resize(B.ps.size());
  for (size_t r = 0; r < B.ps.size(); ++r) {
    for (auto &a : live_arrays(B.ps[r])) {
      void *c = nullptr;
      cudaError_t e = dev_alloc(&c, a.second);
      if (e != cudaSuccess) return e;
      bk.bufs[r].push_back({c, a.second});
      if ((e = cudaMemcpyAsync(c, a.first, a.second, cudaMemcpyDeviceToDevice, st)) != cudaSuccess)
        return e;
    }
  }
  return cudaSuccess;
}

cudaError_t restore_state(Batch &B, Backup &bk, cudaStream_t st) {
  for (size_t r = 0; r < B.ps.size(); ++r) {
    const auto live = live_arrays(B.ps[r]);
    for (size_t q = 0; q < live.size(); ++q) {
      cudaError_t e = cudaMemcpyAsync(live[q].first, bk.bufs[r][q].first, live[q].second,
                                      cudaMemcpyDeviceToDevice, st);
      if (e != cudaSuccess) return e;
    }
  }
  return cudaSuccess;
}

std::string tune_key(const Batch &B) {
  cudaDeviceProp prop;
  int dev = 0;
  cudaGetDevice(&dev);
  cudaGetDeviceProperties(&prop, dev);
  std::ostringstream k;
  int64_t n = 0;
  for (pg_pset *p : B.ps) n += p->n;
  k << prop.name << "|grid " << B.fs->nx << "x" << B.fs->ny << "x" << B.fs->nz << "|storage "
    << B.fs->storage << "|releases " << B.ps.size() << "|particles " << n << "|window "
    << B.window;
  return k.str();
}

bool read_cache(const char *path, const std::string &key, pg_tune &t) {
  if (!path) return false;
  std::ifstream f(path);
  std::string line;
  while (std::getline(f, line)) {
    const size_t bar = line.rfind('\t');
    if (bar == std::string::npos || line.substr(0, bar) != key) continue;
    if (sscanf(line.c_str() + bar + 1, "%d %d", &t.block, &t.resort_steps) == 2) return true;
  }
  return false;
}

void write_cache(const char *path, const std::string &key, const pg_tune &t) {
  if (!path) return;
  std::ofstream f(path, std::ios::app);
  f << key << '\t' << t.block << ' ' << t.resort_steps << '\n';
}

}  // namespace

}  // namespace pg

using namespace pg;

#define CUB(call)                                                                     \
  do {                                                                                \
    cudaError_t e_ = (call);                                                          \
    if (e_ != cudaSuccess) {                                                          \
      set_error("%s failed: %s", #call, cudaGetErrorString(e_));                      \
      return e_ == cudaErrorMemoryAllocation ? PG_ERR_NOMEM : PG_ERR_CUDA;            \
    }                                                                                 \
  } while (0)

extern "C" pg_status pg_execute_batch(int nrel, pg_pset *const *psets,
                                      const pg_kernel *const *kernels, const double *runtime,
                                      const double *dt, double window, const pg_tune *tune,
                                      pg_tune *chosen, const char *tune_cache, int use_graph,
                                      void *stream, int64_t *steps_done) {
  clear_error();
  if (nrel <= 0 || !psets || !kernels || !runtime || !dt) {
    set_error("invalid argument: need nrel > 0 and the release arrays");
    return PG_ERR_ARG;
  }
  if (!(window > 0.0) || !std::isfinite(window)) {
    set_error("invalid argument: window must be > 0");
    return PG_ERR_ARG;
  }
  if (tune && (tune->block < 32 || tune->block > 256 || tune->block % 32 || tune->resort_steps < 0)) {
    set_error("invalid argument: tune.block must be a multiple of 32 in [32, 256], "
              "tune.resort_steps (windows between re-sorts) >= 0");
    return PG_ERR_ARG;
  }
  Batch B;
  B.fs = psets[0] ? psets[0]->fs : nullptr;
  B.window = window;
  double t_begin = 1e300, t_end_max = -1e300;
  for (int r = 0; r < nrel; ++r) {
    pg_pset *p = psets[r];
    if (!p || !kernels[r] || p->fs != B.fs) {
      set_error("invalid argument: release %d has no particle set, no kernel, or another field set", r);
      return PG_ERR_ARG;
    }
    if (p->pos != PG_POS_F32) {
      set_error("batched execution needs FP32 lon/lat/depth positions (release %d)", r);
      return PG_ERR_UNSUPPORTED;
    }
    if (!(dt[r] > 0.0) || !std::isfinite(dt[r]) || !(runtime[r] >= 0.0)) {
      set_error("invalid argument: release %d needs dt > 0 and runtime >= 0", r);
      return PG_ERR_ARG;
    }
    t_begin = std::min(t_begin, p->t_min);
    t_end_max = std::max(t_end_max, p->t_min + runtime[r]);
  }
  pg_fieldset *fs = B.fs;
  if (fs->interp != PG_LINEAR) {
    set_error("batched execution interpolates linearly");
    return PG_ERR_UNSUPPORTED;
  }
  for (int r = 0; r < nrel; ++r)
    if ((kernels[r]->beh & (PG_SETTLE | PG_AGE | PG_SAMPLE)) || kernels[r]->scheme == PG_RKF45) {
      set_error("batched execution runs RK4 or Euler advection, Brownian motion and sinking "
                "only (release %d)", r);
      return PG_ERR_UNSUPPORTED;
    }
  if (fs->streaming || fs->nt < 1) {
    set_error("batched execution needs all snapshots resident");
    return PG_ERR_UNSUPPORTED;
  }
  for (int s = 0; s < fs->nt; ++s)
    if (!fs->slabs[s]) {
      set_error("snapshot %d has not been loaded", s);
      return PG_ERR_STATE;
    }
  if (fs->nt > 1 && fs->period <= 0.0 &&
      (t_begin < fs->times.front() || t_end_max > fs->times.back())) {
    set_error("batch spans [%g, %g] outside the field times", t_begin, t_end_max);
    return PG_ERR_TIME;
  }
  cudaStream_t st = (cudaStream_t)stream;
  B.t_begin = t_begin;
  B.nwin = (int)std::ceil((t_end_max - t_begin) / window - 1e-9);
  if (B.nwin < 1) B.nwin = 1;
  B.ps.assign(psets, psets + nrel);
  // release table and work list (tiles of 32 particles x blocks later: tile
  // length is the block size, so tiles are rebuilt per block size)
  B.rel.resize(nrel);
  std::vector<double> weight(nrel);
  for (int r = 0; r < nrel; ++r) {
    pg_pset *p = psets[r];
    const pg_kernel *k = kernels[r];
    BatchRelease &R = B.rel[r];
    R.p = PartArgs{};
    R.p.n = p->n;
    R.p.x = p->x; R.p.y = p->y; R.p.z = p->z;
    R.p.time = p->time; R.p.id = p->id; R.p.step = p->step; R.p.status = p->status;
    {
      const pg_status rk = resolve_kernel(k, fs, p->seed, R.k);
      if (rk) return rk;
    }
    R.dt = dt[r];
    R.t_end = p->t_min + runtime[r];
    weight[r] = (double)(k->scheme == PG_RK4 ? 4 : 1) * std::min(window, runtime[r]) / dt[r] *
                ((k->beh & PG_BROWNIAN) ? 1.3 : 1.0);
  }
  CUB(dev_alloc((void **)&B.d_rel, sizeof(BatchRelease) * nrel));
  CUB(cudaMemcpy(B.d_rel, B.rel.data(), sizeof(BatchRelease) * nrel, cudaMemcpyHostToDevice));
  CUB(dev_alloc((void **)&B.d_next, sizeof(int) * B.nwin));
  CUB(dev_alloc((void **)&B.d_steps, 8));
  CUB(dev_alloc((void **)&B.d_err, 4));
  std::vector<int> order(nrel);
  for (int r = 0; r < nrel; ++r) order[r] = r;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return weight[a] > weight[b]; });
  auto build_tiles = [&](int block) -> pg_status {
    std::vector<int2> tiles;
    for (int r : order)
      for (int64_t off = 0; off < psets[r]->n; off += block) tiles.push_back(make_int2(r, (int)off));
    dev_free(B.d_tiles);
    B.d_tiles = nullptr;
    B.ntiles = (int)tiles.size();
    CUB(dev_alloc((void **)&B.d_tiles, sizeof(int2) * std::max<size_t>(tiles.size(), 1)));
    if (!tiles.empty())
      CUB(cudaMemcpy(B.d_tiles, tiles.data(), sizeof(int2) * tiles.size(), cudaMemcpyHostToDevice));
    return PG_OK;
  };
  for (pg_pset *p : B.ps)
    if (p->n >= kResortMin) CUB(prepare_resort(p));

  // ------------------------------------------------------------ autotune
  pg_tune use{128, 1, 0};
  if (tune) {
    use = *tune;
  } else {
    const std::string key = tune_key(B);
    if (!read_cache(tune_cache, key, use)) {
      Backup bk;
      CUB(save_state(B, bk, st));
      const int trial = std::min(B.nwin, 4);
      const int blocks[] = {64, 128, 256};
      // never; before the first window and every 1, 2 or 4 windows; before the
      // first window only (an interval of the whole run)
      const int last = std::max(B.nwin, 5);
      const int resorts[] = {0, 1, 2, 4, last};
      // The sort before the first window is paid once per run and its gain
      // lasts the whole run, so a trial charges it at the share of the run
      // the trial covers (trial / nwin of its time).
      float best = 1e30f;
      cudaEvent_t e0, e1, e2;
      CUB(cudaEventCreate(&e0));
      CUB(cudaEventCreate(&e1));
      CUB(cudaEventCreate(&e2));
      for (int bl : blocks)
        for (int rs : resorts) {
          if (build_tiles(bl)) {
            cudaEventDestroy(e0); cudaEventDestroy(e1); cudaEventDestroy(e2);
            return PG_ERR_CUDA;
          }
          CUB(restore_state(B, bk, st));
          CUB(cudaMemsetAsync(B.d_next, 0, sizeof(int) * B.nwin, st));
          CUB(cudaEventRecord(e0, st));
          if (rs > 0) CUB(sort_releases(B, st));
          CUB(cudaEventRecord(e1, st));
          CUB(enqueue_windows(B, 0, trial, bl, rs, st, false));
          CUB(cudaEventRecord(e2, st));
          CUB(cudaEventSynchronize(e2));
          float ms_sort = 0.f, ms_win = 0.f;
          CUB(cudaEventElapsedTime(&ms_sort, e0, e1));
          CUB(cudaEventElapsedTime(&ms_win, e1, e2));
          const float ms = ms_win + ms_sort * (float)trial / (float)B.nwin;
          if (ms < best) { best = ms; use.block = bl; use.resort_steps = rs; }
        }
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      cudaEventDestroy(e2);
      CUB(restore_state(B, bk, st));
      CUB(cudaStreamSynchronize(st));
      write_cache(tune_cache, key, use);
    }
  }
  if (chosen) *chosen = use;
  if (build_tiles(use.block)) return PG_ERR_CUDA;

  // ------------------------------------------------------------ the run
  CUB(cudaMemsetAsync(B.d_next, 0, sizeof(int) * B.nwin, st));
  CUB(cudaMemsetAsync(B.d_steps, 0, 8, st));
  CUB(cudaMemsetAsync(B.d_err, 0, 4, st));
  if (use_graph) {
    // capture on a stream of our own (the legacy stream cannot capture),
    // ordered after the caller's stream and before its later work
    cudaStream_t cap;
    CUB(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
    cudaEvent_t ev;
    CUB(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    CUB(cudaEventRecord(ev, st));
    CUB(cudaStreamWaitEvent(cap, ev, 0));
    cudaGraph_t graph = nullptr;
    CUB(cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = enqueue_windows(B, 0, B.nwin, use.block, use.resort_steps, cap);
    cudaError_t e2 = cudaStreamEndCapture(cap, &graph);
    if (e != cudaSuccess || e2 != cudaSuccess) {
      if (graph) cudaGraphDestroy(graph);
      cudaStreamDestroy(cap);
      cudaEventDestroy(ev);
      set_error("graph capture failed: %s", cudaGetErrorString(e != cudaSuccess ? e : e2));
      return PG_ERR_CUDA;
    }
    cudaGraphExec_t exec = nullptr;
    e = cudaGraphInstantiate(&exec, graph, 0);
    if (e == cudaSuccess) e = cudaGraphLaunch(exec, cap);
    if (e == cudaSuccess) e = cudaEventRecord(ev, cap);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(st, ev, 0);
    if (e == cudaSuccess) e = cudaStreamSynchronize(cap);
    if (exec) cudaGraphExecDestroy(exec);
    cudaGraphDestroy(graph);
    cudaStreamDestroy(cap);
    cudaEventDestroy(ev);
    if (e != cudaSuccess) {
      set_error("graph launch failed: %s", cudaGetErrorString(e));
      return PG_ERR_CUDA;
    }
    note_launches(0);
  } else {
    CUB(enqueue_windows(B, 0, B.nwin, use.block, use.resort_steps, st));
  }
  unsigned long long done = 0;
  int err = 0;
  CUB(cudaMemcpyAsync(&done, B.d_steps, 8, cudaMemcpyDeviceToHost, st));
  CUB(cudaMemcpyAsync(&err, B.d_err, 4, cudaMemcpyDeviceToHost, st));
  CUB(cudaStreamSynchronize(st));
  if (steps_done) *steps_done = (int64_t)done;
  for (int r = 0; r < nrel; ++r) {
    pg_pset *p = psets[r];
    const double te = B.rel[r].t_end;
    p->t_min = std::max(p->t_min, te);
    p->t_max = std::max(p->t_max, te);
  }
  if (err) {
    set_error("a kernel recorded internal error %d", err);
    return PG_ERR_DEVICE;
  }
  return PG_OK;
}
