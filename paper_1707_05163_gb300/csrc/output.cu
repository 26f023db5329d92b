// output.cu -- trajectory output at output times (the ParticleFile of
// Sect. 3) through a pinned two-slot ring, overlapped with the next launch.
//
// At an output time the compute stream packs the rows of the output into a
// device slot: every particle (complete mode) or, in the indexed form of
// Sect. 3, only the particles alive at that time and those deleted since the
// previous output time (each particle's records end with the record of its
// deletion).  A side stream then copies the slot into pinned host memory
// while the next launch advances the particles; the caller's callback for
// output k runs on the host when output k + 1 has been packed (or at the end
// of the execute), so neither the copy nor the callback holds up the GPU.
//
// Rows keep the library's particle order (a tile compaction with a
// deterministic scan), positions are widened to FP64 (the cell form is
// turned back into lon/lat/depth), and the particle variables travel with
// them.
#include "pg_host.h"

namespace pg {

namespace {

constexpr int kOutThreads = 1024;
constexpr int kOutItems = 16;
constexpr int64_t kOutTile = (int64_t)kOutThreads * kOutItems;   // rows per block

// Row selection: complete mode takes every particle; the indexed form takes
// the alive ones and the ones whose time is at or past the previous output
// time in the direction of the run (deleted during this interval; a deleted
// particle keeps the time of its last state).
__device__ __forceinline__ bool selected(const uint8_t *status, const double *time, int64_t i,
                                         int indexed, double t_prev, double sgn) {
  if (!indexed) return true;
  return status[i] == 0 || sgn * (time[i] - t_prev) >= 0.0;
}

__global__ void tile_count_kernel(const uint8_t *status, const double *time, int64_t n,
                                  int indexed, double t_prev, double sgn, uint32_t *tile_count) {
  const int64_t base = (int64_t)blockIdx.x * kOutTile;
  uint32_t c = 0;
  for (int k = 0; k < kOutItems; ++k) {
    const int64_t i = base + (int64_t)k * kOutThreads + threadIdx.x;
    if (i < n && selected(status, time, i, indexed, t_prev, sgn)) ++c;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(0xffffffffu, c, o);
  __shared__ uint32_t ws[kOutThreads / 32];
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = c;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t t = 0;
    for (int w = 0; w < kOutThreads / 32; ++w) t += ws[w];
    tile_count[blockIdx.x] = t;
  }
}

// Exclusive scan of the tile counts in one block (tiles <= kOutThreads *
// kOutItems), total into *count.
__global__ void tile_scan_kernel(const uint32_t *tile_count, int64_t tiles, uint32_t *tile_off,
                                 uint32_t *count) {
  __shared__ uint32_t s[kOutThreads];
  const int64_t per = (tiles + kOutThreads - 1) / kOutThreads;
  const int64_t b0 = (int64_t)threadIdx.x * per;
  uint32_t local = 0;
  for (int64_t b = b0; b < b0 + per && b < tiles; ++b) local += tile_count[b];
  s[threadIdx.x] = local;
  __syncthreads();
  for (int o = 1; o < kOutThreads; o <<= 1) {
    const uint32_t add = threadIdx.x >= (unsigned)o ? s[threadIdx.x - o] : 0u;
    __syncthreads();
    s[threadIdx.x] += add;
    __syncthreads();
  }
  uint32_t run = s[threadIdx.x] - local;
  for (int64_t b = b0; b < b0 + per && b < tiles; ++b) {
    tile_off[b] = run;
    run += tile_count[b];
  }
  if (threadIdx.x == kOutThreads - 1) *count = s[threadIdx.x];
}

struct PackArgs {
  GridArgs g;
  int pos;                       // PG_POS_*
  const void *x, *y, *z;
  const int32_t *ci, *cj, *ck;
  const float *fx, *fy, *fz;
  const double *time, *age, *var;
  const uint64_t *id;
  const uint8_t *status;
  int64_t n, vstride;
  int nvar, indexed;
  double t_prev, sgn;
  const uint32_t *tile_off;
  // slot arrays, cap rows each
  uint64_t *o_id;
  double *o_lon, *o_lat, *o_dep, *o_age, *o_var;
  uint8_t *o_status;
  int64_t cap;
};

// Each block compacts its tile in order: a block-wide scan of the selected
// flags (thread-major within a pass over kOutThreads rows), offset by the
// tile's start.
__global__ void pack_kernel(const PackArgs a) {
  __shared__ uint32_t ws[kOutThreads / 32];
  __shared__ uint32_t pass_base;
  const int64_t base = (int64_t)blockIdx.x * kOutTile;
  if (threadIdx.x == 0) pass_base = a.tile_off[blockIdx.x];
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int k = 0; k < kOutItems; ++k) {
    const int64_t i = base + (int64_t)k * kOutThreads + threadIdx.x;
    const bool sel = i < a.n && selected(a.status, a.time, i, a.indexed, a.t_prev, a.sgn);
    const unsigned m = __ballot_sync(0xffffffffu, sel);
    if (lane == 0) ws[warp] = __popc(m);
    __syncthreads();
    uint32_t before = 0, total = 0;
    for (int w = 0; w < kOutThreads / 32; ++w) {
      const uint32_t c = ws[w];
      if (w < warp) before += c;
      total += c;
    }
    const uint32_t o = pass_base + before + __popc(m & ((1u << lane) - 1u));
    if (sel) {
      double lon, lat, dep;
      if (a.pos == PG_POS_F64) {
        lon = ((const double *)a.x)[i]; lat = ((const double *)a.y)[i];
        dep = ((const double *)a.z)[i];
      } else if (a.pos == PG_POS_F32) {
        lon = ((const float *)a.x)[i]; lat = ((const float *)a.y)[i];
        dep = ((const float *)a.z)[i];
      } else {
        // the same rounding as pg_pset_get's conversion (one fused multiply-add)
        lon = __fma_rn((double)a.ci[i] + (double)a.fx[i], a.g.d[0], a.g.x0[0]);
        lat = __fma_rn((double)a.cj[i] + (double)a.fy[i], a.g.d[1], a.g.x0[1]);
        dep = a.g.nz > 1 ? __fma_rn((double)a.ck[i] + (double)a.fz[i], a.g.d[2], a.g.x0[2]) : 0.0;
      }
      a.o_id[o] = a.id[i];
      a.o_lon[o] = lon; a.o_lat[o] = lat; a.o_dep[o] = dep;
      a.o_status[o] = a.status[i];
      a.o_age[o] = a.age[i];
      for (int j = 0; j < a.nvar; ++j) a.o_var[(int64_t)j * a.cap + o] = a.var[(int64_t)j * a.vstride + i];
    }
    __syncthreads();
    if (threadIdx.x == 0) pass_base += total;
    __syncthreads();
  }
}

}  // namespace

// Bytes of one slot for `cap` rows and `nvar` variables: id, lon, lat,
// depth, age, vars (8 bytes each), status (1 byte), the row count.
static size_t slot_bytes(int64_t cap, int nvar) {
  return (size_t)cap * (8 * (5 + (size_t)nvar) + 1) + 16;
}

OutputRing::~OutputRing() { release(); }

void OutputRing::release() {
  for (auto &s : slot) {
    dev_free(s.d);
    if (s.h) cudaFreeHost(s.h);
    if (s.packed) cudaEventDestroy(s.packed);
    if (s.copied) cudaEventDestroy(s.copied);
    s = OutputSlot();
  }
  dev_free(d_tiles);
  d_tiles = nullptr;
  if (cs) cudaStreamDestroy(cs);
  cs = nullptr;
  cap = 0;
}

cudaError_t OutputRing::prepare(int64_t need_cap, int need_nvar) {
  if (cap >= need_cap && nvar == need_nvar && cs) return cudaSuccess;
  release();
  const size_t bytes = slot_bytes(need_cap, need_nvar);
  const int64_t tiles = (need_cap + kOutTile - 1) / kOutTile;
  cudaError_t e = cudaSuccess;
  for (auto &s : slot) {
    if (e == cudaSuccess) e = dev_alloc(&s.d, bytes);
    if (e == cudaSuccess) e = cudaMallocHost(&s.h, bytes);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s.packed, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s.copied, cudaEventDisableTiming);
  }
  if (e == cudaSuccess) e = dev_alloc((void **)&d_tiles, sizeof(uint32_t) * 2 * (size_t)(tiles + 1));
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    release();
    return e;
  }
  cap = need_cap;
  nvar = need_nvar;
  next = 0;
  return cudaSuccess;
}

// Views of a slot's arrays (device or host base).
OutputView OutputRing::view(const void *base, int64_t rows_cap, int nv) {
  OutputView v;
  char *p = (char *)base;
  v.id = (uint64_t *)p; p += rows_cap * 8;
  v.lon = (double *)p; p += rows_cap * 8;
  v.lat = (double *)p; p += rows_cap * 8;
  v.depth = (double *)p; p += rows_cap * 8;
  v.age = (double *)p; p += rows_cap * 8;
  v.vars = (double *)p; p += rows_cap * 8 * nv;
  v.status = (uint8_t *)p; p += rows_cap;
  v.count = (uint32_t *)(((uintptr_t)p + 7) & ~(uintptr_t)7);
  return v;
}

cudaError_t OutputRing::enqueue(const pg_pset *ps, double t, double t_prev, double sgn,
                                int indexed, cudaStream_t st) {
  OutputSlot &s = slot[next];
  const int64_t n = ps->n;
  const int64_t tiles = n > 0 ? (n + kOutTile - 1) / kOutTile : 0;
  if (tiles > kOutTile) return cudaErrorInvalidValue;
  uint32_t *tile_count = d_tiles, *tile_off = d_tiles + tiles + 1;
  OutputView dv = view(s.d, cap, nvar);
  cudaError_t e;
  if (tiles > 0) {
    tile_count_kernel<<<(unsigned)tiles, kOutThreads, 0, st>>>(ps->status, ps->time, n, indexed,
                                                               t_prev, sgn, tile_count);
    tile_scan_kernel<<<1, kOutThreads, 0, st>>>(tile_count, tiles, tile_off, dv.count);
    PackArgs a;
    a.g = grid_args_of(ps->fs);
    a.pos = ps->pos;
    a.x = ps->x; a.y = ps->y; a.z = ps->z;
    a.ci = ps->ci; a.cj = ps->cj; a.ck = ps->ck;
    a.fx = ps->fx; a.fy = ps->fy; a.fz = ps->fz;
    a.time = ps->time; a.age = ps->age; a.var = ps->var;
    a.id = ps->id; a.status = ps->status;
    a.n = n; a.vstride = ps->cap; a.nvar = nvar; a.indexed = indexed;
    a.t_prev = t_prev; a.sgn = sgn; a.tile_off = tile_off;
    a.o_id = dv.id; a.o_lon = dv.lon; a.o_lat = dv.lat; a.o_dep = dv.depth;
    a.o_age = dv.age; a.o_var = dv.vars; a.o_status = dv.status; a.cap = cap;
    pack_kernel<<<(unsigned)tiles, kOutThreads, 0, st>>>(a);
    note_launches(3);
  } else if ((e = cudaMemsetAsync(dv.count, 0, 4, st)) != cudaSuccess) {
    return e;
  }
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if ((e = cudaEventRecord(s.packed, st)) != cudaSuccess) return e;
  // the copy runs on the side stream while the compute stream goes on
  if ((e = cudaStreamWaitEvent(cs, s.packed, 0)) != cudaSuccess) return e;
  if ((e = cudaMemcpyAsync(s.h, s.d, slot_bytes(cap, nvar), cudaMemcpyDeviceToHost, cs)) !=
      cudaSuccess)
    return e;
  if ((e = cudaEventRecord(s.copied, cs)) != cudaSuccess) return e;
  s.time = t;
  s.pending = true;
  next ^= 1;
  return cudaSuccess;
}

cudaError_t OutputRing::wait(int k, OutputView &hv, double &t) {
  OutputSlot &s = slot[k];
  const cudaError_t e = cudaEventSynchronize(s.copied);
  if (e != cudaSuccess) return e;
  hv = view(s.h, cap, nvar);
  t = s.time;
  return cudaSuccess;
}

}  // namespace pg
