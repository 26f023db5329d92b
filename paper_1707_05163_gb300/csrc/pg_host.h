// pg_host.h -- host-side objects behind the C ABI and the kernel launchers.
#pragma once

#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <map>
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
  double *age = nullptr;      // [cap]
  double *var = nullptr;      // [nvar][cap] sampled variables
  double *hstep = nullptr;    // [cap] RKF45 step lengths
  void free_all() {
    void *ps[] = {x, y, z, ci, cj, ck, fx, fy, fz, time, id, step, status, age, var, hstep};
    for (void *p : ps) dev_free(p);
    *this = PsetArrays();
  }
};

// Allocate the arrays of `cap` particles with `nvar` sampled variables.
pg_status alloc_arrays(PsetArrays &A, int pos, int64_t cap, int nvar);

// Arrays of one output slot (device or pinned host), cap rows each.
struct OutputView {
  uint64_t *id = nullptr;
  double *lon = nullptr, *lat = nullptr, *depth = nullptr, *age = nullptr;
  double *vars = nullptr;       // [nvar][cap]
  uint8_t *status = nullptr;
  uint32_t *count = nullptr;    // rows written
};

struct OutputSlot {
  void *d = nullptr;            // device slot
  void *h = nullptr;            // pinned host copy
  cudaEvent_t packed = nullptr, copied = nullptr;
  double time = 0.0;
  bool pending = false;
};

// Two-slot pinned output ring of a particle set (output.cu).
struct OutputRing {
  int64_t cap = 0;
  int nvar = 0;
  OutputSlot slot[2];
  uint32_t *d_tiles = nullptr;  // tile counts and offsets of the compaction
  cudaStream_t cs = nullptr;    // the copy stream
  int next = 0;                 // slot of the next output
  ~OutputRing();
  void release();
  cudaError_t prepare(int64_t need_cap, int need_nvar);
  // pack the output at time t into slot `next` on `st` and copy it to the
  // host on the copy stream; indexed: rows of alive particles and of those
  // deleted at or after t_prev (direction sgn)
  cudaError_t enqueue(const pg_pset *ps, double t, double t_prev, double sgn, int indexed,
                      cudaStream_t st);
  // wait for slot k's copy; host views of its arrays and its time
  cudaError_t wait(int k, OutputView &hv, double &t);
  static OutputView view(const void *base, int64_t rows_cap, int nv);
};

}  // namespace pg

struct pg_fieldset {
  int device = 0;
  // constants carried by the field set (Sect. 3), read by the behaviours
  std::map<std::string, double> constants;
  int interp = 0;               // velocities: 0 linear, 1 nearest
  // scalar fields (tracers) sampled into particle variables, resident only
  int ntr = 0;
  std::string tr_name[2];
  int tr_interp[2] = {0, 0};
  std::vector<void *> tr_slabs; // [2 * nt] planar slabs (null until loaded)
  const void **d_ttab = nullptr;// device copy of tr_slabs
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
  std::vector<pg::Slot> slot = std::vector<pg::Slot>(4);   // the ring (>= 4 slots)
  void *h_pinned = nullptr;     // pinned staging for callback sources
  cudaStream_t side = nullptr;
  cudaEvent_t stage_free = nullptr;
  int64_t uploads = 0;          // streamed snapshot uploads
  int64_t upload_h2d_bytes = 0; // of which host-to-device bytes
};

struct pg_kernel {
  int scheme = PG_RK4;
  unsigned beh = 0;
  double kh = 0.0, w_sink = 0.0;   // NaN: the field set's constant of that name
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
  double *age = nullptr;               // [cap] age in seconds (age behaviour)
  double *var = nullptr;               // [nvar][cap] sampled variables
  double *hstep = nullptr;             // [cap] RKF45 step lengths (0: start from dt)
  int nvar = 0;                        // the field set's scalar fields at creation
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
  // trajectory output ring, on first use
  pg::OutputRing *out = nullptr;
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

// One network step of the learned flow map fused into the tcgen05 inference
// kernel: the particles' features gathered on chip, the network, the
// displacement applied to the particles (surrogate_features.cuh).
struct SurrogateStepIO {
  GridArgs g;
  FieldArgs f;
  float *lon, *lat, *dep;
  double *time;
  uint32_t *step;
  uint8_t *status;
  int64_t n;
  double horizon;
  int *ferr;                  // device word: feature error (time range, missing slab)
};
// Whether the network's engine and shape allow the fused step.
bool mlp_fused_step_ok(const pg_mlp *net);
// The fused step (weights packed first if needed); reads back the network's
// and the features' error words.
pg_status mlp_fused_step(pg_mlp *net, const SurrogateStepIO &io, cudaStream_t st);

// Kernel argument block of a kernel on a field set: NaN parameters and those
// of the settle and age behaviours from the field set's constants (capi.cu).
pg_status resolve_kernel(const pg_kernel *k, const pg_fieldset *fs, uint64_t seed, KernArgs &a);

// The device arrays of a particle set, and replacing them (capi.cu).
PsetArrays pset_arrays(const pg_pset *ps);
void pset_set_arrays(pg_pset *ps, const PsetArrays &A);

// Advection chunk with the worked example's behaviours or nearest-neighbour
// interpolation on FP32 positions and FP32 storage (advect_f32_ext.cu).
cudaError_t launch_advect_plain_ext(const StepArgs &a, int block, cudaStream_t st);

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
