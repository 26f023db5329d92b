// pg_host.h -- host-side objects behind the C ABI and the kernel launchers.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/parcels_gb.h"
#include "pg_device.cuh"

namespace pg {

void set_error(const char *fmt, ...);
void clear_error();

// Every device allocation of the library goes through these two, so the
// accounting (and failure injection in tests) has one place.
cudaError_t dev_alloc(void **p, size_t bytes);
void dev_free(void *p);

// Count of kernel launches made by the library (all threads, all devices).
void note_launches(int n);

struct Slot {
  void *buf = nullptr;        // interleaved slab in storage format
  float *scales = nullptr;    // [nf] FP32 scales of this slot
  int s = -1;                 // snapshot held (-1: none)
  cudaEvent_t ready = nullptr;   // upload finished (recorded on the side stream)
  cudaEvent_t free = nullptr;    // last use finished (recorded on the compute stream)
};

// Device arrays of one particle set (positions in one of the two forms).
struct PsetArrays {
  void *x = nullptr, *y = nullptr, *z = nullptr;
  int32_t *ci = nullptr, *cj = nullptr, *ck = nullptr;
  float *fx = nullptr, *fy = nullptr, *fz = nullptr;
  double *time = nullptr;
  uint64_t *id = nullptr;
  uint32_t *step = nullptr;
  uint8_t *status = nullptr;
  void free_all() {
    void *ps[] = {x, y, z, ci, cj, ck, fx, fy, fz, time, id, step, status};
    for (void *p : ps) dev_free(p);
    *this = PsetArrays();
  }
};

pg_status alloc_arrays(PsetArrays &A, int pos, int64_t cap);

}  // namespace pg

struct pg_fieldset {
  int device = 0;
  int sm_count = 0;
  int nx = 0, ny = 0, nz = 0, mesh = 0, periodic = 0, nfields = 0, storage = 0;
  std::vector<double> lon, lat, depth;
  double *d_axes64 = nullptr;   // lon | lat | depth
  float *d_axes32 = nullptr;
  int uni[3] = {0, 0, 0};
  double x0[3] = {0, 0, 0}, inv_d[3] = {0, 0, 0};
  // time axis
  int nt = 0;
  std::vector<double> times;
  double period = 0.0;
  double *d_times = nullptr;
  // storage
  size_t nodes = 0;             // nx * ny * nz
  size_t slab_bytes = 0;        // interleaved slab in storage format
  std::vector<void *> slabs;    // resident snapshots (null until loaded)
  std::vector<float> h_scales;  // [nt * nf]
  const void **d_tab = nullptr; // device table [nt]
  float *d_scales = nullptr;    // device [nt * nf]
  unsigned *d_amax = nullptr;   // scratch of the quantiser
  void *d_stage = nullptr;      // planar staging buffer (host-sourced uploads)
  size_t stage_bytes = 0;
  // streaming
  bool streaming = false;
  std::vector<const void *> src_ptrs;
  pg_snapshot_cb cb = nullptr;
  void *cb_user = nullptr;
  int src_dtype = PG_F32;
  pg::Slot slot[4];
  void *h_pinned = nullptr;     // pinned staging for callback sources
  cudaStream_t side = nullptr;
  cudaEvent_t stage_free = nullptr;
  int64_t uploads = 0;          // streamed snapshot uploads
  int64_t upload_h2d_bytes = 0; // of which host-to-device bytes
};

struct pg_kernel {
  int scheme = PG_RK4;
  unsigned beh = 0;
  double kh = 0.0, w_sink = 0.0;
};

struct pg_pset {
  pg_fieldset *fs = nullptr;
  int pos = PG_POS_F32;
  uint64_t seed = 0;
  int64_t n = 0, cap = 0;
  void *x = nullptr, *y = nullptr, *z = nullptr;       // positions (plain forms)
  int32_t *ci = nullptr, *cj = nullptr, *ck = nullptr;  // cell form
  float *fx = nullptr, *fy = nullptr, *fz = nullptr;
  double *time = nullptr;
  uint64_t *id = nullptr;
  uint32_t *step = nullptr;
  uint8_t *status = nullptr;
  double t_min = 0.0, t_max = 0.0;     // range of particle times
  pg_tune tune{256, 0, 64};
  unsigned long long *d_counter = nullptr;
  int *d_err = nullptr;
  // re-sort: second set of arrays (same capacity) and scratch, on first use
  pg::PsetArrays alt;
  int64_t alt_cap = 0;
  void *sort_scratch = nullptr;
  size_t sort_scratch_bytes = 0;
  double *diag_scratch = nullptr;
  // optional CUDA-event timing of the advection launches
  bool timing = false;
  std::vector<cudaEvent_t> ev;        // pairs (start, stop) per launch
  size_t ev_used = 0;
  double timed_ms = 0.0;
  int64_t timed_launches = 0;
};

namespace pg {

cudaError_t launch_repack(const void *src, int src_dtype, int nf, size_t nodes, void *dst,
                          int storage, float *scales_out, unsigned *amax_scratch, int sm_count,
                          cudaStream_t st);

// Advection chunk for lon/lat/depth positions.  real: PG_POS_F64 / PG_POS_F32.
cudaError_t launch_advect_plain(const StepArgs &a, int real, int storage, int block,
                                cudaStream_t st);

// Advection chunk for cell-index + offset positions.
cudaError_t launch_advect_cell(const StepArgs &a, int storage, int block, cudaStream_t st);
cudaError_t launch_to_cell(const GridArgs &g, const double *lon, const double *lat,
                           const double *dep, int32_t *ci, int32_t *cj, int32_t *ck, float *fx,
                           float *fy, float *fz, int64_t n, int sm, cudaStream_t st);
cudaError_t launch_from_cell(const GridArgs &g, const int32_t *ci, const int32_t *cj,
                             const int32_t *ck, const float *fx, const float *fy, const float *fz,
                             double *lon, double *lat, double *dep, int64_t n, int sm,
                             cudaStream_t st);

// Grid argument block of a field set (defined in capi.cu).
GridArgs grid_args_of(const pg_fieldset *fs);

// Element size of one position coordinate for a position form.
inline size_t pos_elem(int pos) { return pos == PG_POS_F64 ? 8 : 4; }
inline size_t storage_elem(int storage) {
  return storage == PG_F64 ? 8 : (storage == PG_F32 ? 4 : 2);
}

}  // namespace pg

namespace pg {

// Geometry kind of a grid; the FP32 kernels are compiled once per kind.
inline int geo_of(const GridArgs &g) {
  return g.mesh != 1 ? GEO_FLAT : (g.periodic ? GEO_SPH_PER : GEO_SPH);
}

// Launch a chunk kernel over a.p.n particles, one thread each.  The block
// size is clamped to what the kernel's register use allows (queried once per
// kernel).
template <void (*Kernel)(StepArgs)>
inline cudaError_t launch_clamped(const StepArgs &a, int block, cudaStream_t st) {
  static int max_threads = 0;
  if (max_threads == 0) {
    cudaFuncAttributes at;
    const cudaError_t e = cudaFuncGetAttributes(&at, Kernel);
    if (e != cudaSuccess) return e;
    max_threads = at.maxThreadsPerBlock;
  }
  const int b = block > max_threads ? (max_threads / 32) * 32 : block;
  const int64_t grid = (a.p.n + b - 1) / b;
  Kernel<<<(unsigned)grid, b, 0, st>>>(a);
  note_launches(1);
  return cudaGetLastError();
}

}  // namespace pg
