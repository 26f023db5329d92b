/*
 * parcels_gb.h -- C ABI of the GB300 particle-advection library.
 *
 * The library advects many independent virtual particles through gridded
 * velocity fields (Lange & van Sebille, "Parcels v0.9", arXiv 1707.05163):
 * each step integrates Eq. 1 with RK4 (default) or Euler-forward (Sect.
 * 2.1.1), sampling U, V[, W] by bi/trilinear interpolation in space and linear
 * interpolation in time on a rectilinear grid (Sect. 2.3, 2.4), then applies
 * composable behaviours -- Brownian motion with uniform K_h (Sect. 2.1.2,
 * 4.2.7) and constant sinking (the behaviour term of Eq. 1) -- a periodic
 * zonal boundary and deletion of particles that leave the domain (the
 * out-of-bounds recovery of Sect. 2.1.2 and 3).  The objects follow the
 * paper's FieldSet / ParticleSet / Kernel / execute statement of the problem
 * (Sect. 2.1, 2.2, 3; Fig. 2).
 *
 * Conventions for every call:
 *   - Return value: PG_OK (0) or a negative PG_ERR_* code.  On error the
 *     objects are left as they were before the call, and pg_last_error()
 *     returns a message for the calling thread.  No call throws or aborts.
 *   - Pointers named "host or device" may point to host memory (pageable or
 *     pinned) or to device memory of the current CUDA device; the library
 *     copies from them during the call (unified addressing).  The caller keeps
 *     ownership of everything it passes in; the library owns what it creates
 *     and frees it in the matching pg_*_destroy.
 *   - `stream` is a cudaStream_t (NULL = the legacy default stream).  All
 *     device work of a call is ordered on it; calls return after the work
 *     they launched has completed unless stated otherwise.
 *   - Units: flat mesh positions in metres; spherical mesh lon/lat in degrees;
 *     depth in metres, positive downward; velocities in m/s (W positive
 *     downward); times and dt in seconds.
 */
#ifndef PARCELS_GB_H
#define PARCELS_GB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int pg_status;

/* Symbols of this header are exported from the shared library. */
#if defined(__GNUC__)
#define PG_API __attribute__((visibility("default")))
#else
#define PG_API
#endif

/* Error codes. */
#define PG_OK 0
#define PG_ERR_ARG (-1)         /* invalid argument; nothing changed            */
#define PG_ERR_CUDA (-2)        /* a CUDA call failed                           */
#define PG_ERR_STATE (-3)       /* call not valid in the object's current state */
#define PG_ERR_TIME (-4)        /* time span outside the field's time range     */
#define PG_ERR_CALLBACK (-5)    /* a user callback returned non-zero            */
#define PG_ERR_TIMEOUT (-6)     /* a bounded device wait gave up                */
#define PG_ERR_NOMEM (-7)       /* device or host allocation failed             */
#define PG_ERR_UNSUPPORTED (-8) /* combination of options not implemented       */
#define PG_ERR_DEVICE (-9)      /* a kernel recorded an internal check failure  */

/* Mesh (Sect. 4.2.2): flat (metres) or spherical (degrees, converted with
 * 1852*60 metres per degree of latitude, and per degree of longitude times
 * the cosine of latitude). */
#define PG_FLAT 0
#define PG_SPHERICAL 1

/* Field storage in device memory.  F16S/BF16S store binary16/bfloat16 codes
 * with one FP32 scale per (field, snapshot): scale = max|v| / 32752,
 * code = round-to-nearest-even(v / scale), value = code * scale. */
#define PG_F64 0
#define PG_F32 1
#define PG_F16S 2
#define PG_BF16S 3

/* Particle position representation.  F64/F32: lon, lat, depth.  CELL: an
 * int32 cell index per axis plus an FP32 offset in [0, 1) inside the cell
 * (requires uniformly spaced axes). */
#define PG_POS_F64 0
#define PG_POS_F32 1
#define PG_POS_CELL 2

/* Time-stepping scheme (Sect. 2.1.1).  PG_RKF45: adaptive Runge-Kutta-
 * Fehlberg 4(5); each particle keeps its own step length (starting from the
 * execute's |dt|, at most the field set constant "rkf45_max_dt" (default
 * |dt|), at least "rkf45_min_dt" (default 1 s)); a trial whose error (the
 * largest of |X5 - X4| over the axes, in metres) exceeds "rkf45_tol" (metres,
 * required) is repeated at half the length; an accepted step with a tenth of
 * the tolerance doubles the length; steps land on output times and the end
 * time; the particle moves to the fourth-order X4.  Needs lon/lat/depth
 * positions and FP32 or FP64 storage (PG_POS_F32 with PG_F32), outside
 * pg_execute_batch. */
#define PG_EULER 0
#define PG_RK4 1
#define PG_RKF45 2

/* Behaviour bits, applied after advection in this order.  SETTLE, AGE and
 * SAMPLE are the custom kernels of the paper's worked example (Sect. 3; the
 * backward run of virtual foraminifera): their parameters are constants of
 * the field set (pg_fieldset_add_constant).
 *   BROWNIAN: each horizontal coordinate += sqrt(2 Kh |dt|) N(0, 1).
 *   SINK:     depth += w_sink dt.
 *   SETTLE:   while the depth at the start of a step differs from the
 *             constant "dwelling_depth", depth += w_sink dt, stopping at the
 *             dwelling depth when it reaches or passes it; a step that starts
 *             at the dwelling depth holds it (vertical advection discarded).
 *   AGE:      age += |dt| per step (with SETTLE: per step that starts at the
 *             dwelling depth); a particle whose age reaches the constant
 *             "max_age" is deleted with status PG_DELETED after its step.
 *   SAMPLE:   every scalar field of the field set (pg_fieldset_add_scalar)
 *             is interpolated at the particle's position and time after the
 *             step into the particle's variable (pg_pset_get_variables).
 * SETTLE, AGE, SAMPLE and nearest-neighbour interpolation need lon/lat/depth
 * positions (PG_POS_F64, or PG_POS_F32 on PG_F32 storage) and run outside
 * pg_execute_batch. */
#define PG_BROWNIAN 1u
#define PG_SINK 2u
#define PG_SETTLE 4u
#define PG_AGE 8u
#define PG_SAMPLE 16u

/* Spatial interpolation of a field (Sect. 2.3): linear (bi/trilinear), or
 * the nearest node on each axis (the lower node on a tie).  Time is always
 * linear. */
#define PG_LINEAR 0
#define PG_NEAREST 1

/* Particle status (one byte per particle).  Any non-zero status means the
 * particle was deleted; its position and time are those before the step
 * that would have taken it out of the domain. */
#define PG_ALIVE 0
#define PG_OOB_HORIZ 1 /* a stage or final position left the lon/lat range */
#define PG_OOB_DEPTH 2 /* a stage or final position left the depth range   */
#define PG_NAN 3       /* a sampled velocity was NaN                        */
#define PG_DELETED 4   /* deleted by the AGE behaviour (state after its step) */

typedef struct pg_fieldset pg_fieldset;
typedef struct pg_pset pg_pset;
typedef struct pg_kernel pg_kernel;

/* Rectilinear grid (Sect. 2.4): each axis depends on one coordinate only.
 * lon[nx], lat[ny], depth[nz] strictly increasing, host memory, copied.
 * nz == 1 makes a two-dimensional field (depth ignored by the sampling). */
typedef struct {
    int nx, ny, nz;
    const double *lon, *lat, *depth;
} pg_grid;

/* Tuning of the time loop.  Zero fields take defaults. */
typedef struct {
    int block;          /* threads per block of the advection kernel (default 256)  */
    int resort_steps;   /* Morton re-sort before the first launch of an execute and
                           every this many steps (0: never)                          */
    int chunk_steps;    /* at most this many steps per kernel launch (default 64)    */
} pg_tune;

/* Snapshot source for streamed fields (the counterpart of advancing the
 * resident time slices, Sect. 3).  Fill `dst` (host, pinned, `bytes` long)
 * with snapshot `s` laid out [nfields][nz][ny][nx] in the source dtype given
 * to pg_fieldset_stream.  Return 0 on success; non-zero aborts the execute
 * with PG_ERR_CALLBACK. */
typedef int (*pg_snapshot_cb)(void *user, int s, void *dst, size_t bytes);

/* Output hook, called at every output time (the ParticleFile of Sect. 3)
 * with every particle of the set.  Arrays are host memory (pinned, owned by
 * the library) valid during the call only, n entries in the library's
 * internal order (use `id` to match particles).  The hook for output time t
 * runs on the calling thread while the GPU already advances the particles
 * past t (at the next output time or at the end of the execute), so the copy
 * and the hook overlap the computation.  Non-zero return aborts the execute
 * with PG_ERR_CALLBACK. */
typedef int (*pg_output_cb)(void *user, double time, int64_t n, const uint64_t *id,
                            const double *lon, const double *lat, const double *depth,
                            const uint8_t *status);

/* One output record set (pg_execute_records): n rows, library order, host
 * memory valid during the hook only.  Row i: particle id[i] at lon[i],
 * lat[i], depth[i] (FP64), status[i], age[i] and its sampled variables
 * vars[j * var_stride + i], j < nvar. */
typedef struct {
    double time;
    int64_t n;
    int nvar;
    int64_t var_stride;
    const uint64_t *id;
    const double *lon, *lat, *depth;
    const uint8_t *status;
    const double *age;
    const double *vars;
} pg_record;
typedef int (*pg_record_cb)(void *user, const pg_record *rec);

/* ---------------------------------------------------------------- errors */

/* Message describing the last error on the calling thread ("" if none). */
PG_API const char *pg_last_error(void);

/* Library version string. */
PG_API const char *pg_version(void);

/* -------------------------------------------------------------- fieldset */

/* Create a field set (the FieldSet of Sect. 2.4) on the current CUDA device.
 * nfields: 2 (U, V) or 3 (U, V, W; needs nz > 1).  periodic_lon requires a
 * spherical mesh whose lon axis spans less than 360 degrees; the wrap cell
 * joins the last node to the first.  storage: PG_F64, PG_F32, PG_F16S,
 * PG_BF16S.  The field holds no data until snapshots are given. */
PG_API pg_status pg_fieldset_create(const pg_grid *grid, int mesh, int periodic_lon, int nfields,
                             int storage, pg_fieldset **out);

/* Snapshot times (strictly increasing, host memory, nt >= 1; nt == 1 is a
 * steady field).  period > 0 makes the field repeat with that period: after
 * the last snapshot it interpolates towards the first at times[0] + period.
 * Must be called before any snapshot is given; resets existing data. */
PG_API pg_status pg_fieldset_set_times(pg_fieldset *fs, int nt, const double *times, double period);

/* Give snapshot s (host or device memory, [nfields][nz][ny][nx], lon
 * fastest, src_dtype PG_F64 or PG_F32).  The library converts it to its
 * storage format in device memory it owns (all snapshots resident). */
PG_API pg_status pg_fieldset_load_snapshot(pg_fieldset *fs, int s, const void *data, int src_dtype,
                                    void *stream);

/* Stream snapshots instead of keeping them all resident: the library keeps
 * a ring of device slots (four unless pg_fieldset_set_ring says otherwise)
 * and, during pg_execute, uploads the next snapshots on its own side stream
 * while the current ones are in use.  Source: either `ptrs`
 * (nt host or device pointers, each valid for the lifetime of the field
 * set), or `cb` (called with a pinned host buffer to fill).  Exactly one of
 * ptrs / cb must be non-NULL. */
PG_API pg_status pg_fieldset_stream(pg_fieldset *fs, const void *const *ptrs, pg_snapshot_cb cb,
                             void *user, int src_dtype);

/* Size of the streamed-snapshot ring, before pg_fieldset_stream: `slots`
 * device slots of one snapshot each, 4 (default: two snapshots in use by a
 * launch, the third for steps that reach past its end, the next one
 * uploading; the three time slices of Sect. 3 plus the prefetch) to 64.  A
 * launch spans at most B = (slots - 4) / 2 snapshot times after the next one
 * and holds B + 3 slots; the others prefetch the snapshots that follow, in
 * order, so larger rings allow longer launches, at slots x (snapshot bytes)
 * of device memory, without waiting for uploads. */
PG_API pg_status pg_fieldset_set_ring(pg_fieldset *fs, int slots);

/* Device bytes held by the field set's snapshot storage. */
PG_API pg_status pg_fieldset_device_bytes(const pg_fieldset *fs, size_t *bytes);

/* FP32 scale of (field f, snapshot s) for F16S/BF16S storage (1.0 otherwise).
 * Resident storage only. */
PG_API pg_status pg_fieldset_get_scale(const pg_fieldset *fs, int s, int f, float *scale);

/* Named constants of the field set (Sect. 3: the worked example adds three
 * global constants to its FieldSet for its custom kernels).  The behaviours
 * read "Kh" (m^2/s, BROWNIAN when the kernel's kh is NaN), "w_sink" (m/s,
 * SINK and SETTLE when the kernel's w_sink is NaN), "dwelling_depth" (m,
 * SETTLE) and "max_age" (s, AGE) at execute time; other names are kept for
 * the caller.  `name` is copied; values must be finite (PG_ERR_ARG).  Adding
 * a name again replaces its value.  get returns PG_ERR_ARG for an unknown
 * name. */
PG_API pg_status pg_fieldset_add_constant(pg_fieldset *fs, const char *name, double value);
PG_API pg_status pg_fieldset_get_constant(const pg_fieldset *fs, const char *name, double *value);

/* Spatial interpolation of the velocity fields: PG_LINEAR (default) or
 * PG_NEAREST (Sect. 2.3). */
PG_API pg_status pg_fieldset_set_interp(pg_fieldset *fs, int method);

/* Scalar fields on the same grid and snapshot times as the velocities (the
 * temperature field the worked example samples, Sect. 3), at most two per
 * field set, interpolated by `method` (PG_LINEAR / PG_NEAREST) in space and
 * linearly in time.  add: after pg_fieldset_set_times and before the particle
 * sets that sample it are created; *index (may be NULL) receives its number.
 * load: snapshot s of scalar field `index`, [nz][ny][nx] lon fastest, host or
 * device, src_dtype PG_F64 or PG_F32; stored in FP64 for PG_F64 field
 * storage and in FP32 otherwise, resident in device memory the library owns
 * (field sets whose velocities are streamed cannot be sampled).
 * pg_fieldset_set_times drops loaded scalar snapshots. */
PG_API pg_status pg_fieldset_add_scalar(pg_fieldset *fs, const char *name, int method, int *index);
PG_API pg_status pg_fieldset_load_scalar(pg_fieldset *fs, int index, int s, const void *data,
                                         int src_dtype, void *stream);

PG_API pg_status pg_fieldset_destroy(pg_fieldset *fs);

/* ---------------------------------------------------------------- kernel */

/* A composed kernel (Sect. 2.1.2): advection scheme followed by behaviours.
 * kh: Brownian diffusivity in m^2/s (sigma per step sqrt(2 kh |dt|) metres,
 * normal variates from Philox4x32-10 keyed by the particle set's seed and
 * counted by (particle id, particle step)); w_sink: sinking speed in m/s
 * (depth += w_sink * dt).  Either may be NaN: the field set's constant "Kh"
 * or "w_sink" is then used at execute time (PG_ERR_STATE if it is absent). */
PG_API pg_status pg_kernel_create(int scheme, unsigned behaviours, double kh, double w_sink,
                           pg_kernel **out);
PG_API pg_status pg_kernel_destroy(pg_kernel *k);

/* ---------------------------------------------------------- particle set */

/* Create a particle set (the ParticleSet of Sect. 2.1) of n particles on the
 * field set's grid.  lon, lat, depth, time: n doubles each (host or device);
 * depth may be NULL for zero, time may be NULL for t0 everywhere (then
 * `t0` is used).  ids: n uint64 (host or device) or NULL for
 * id_base + 0..n-1.  pos: PG_POS_F64 / PG_POS_F32 / PG_POS_CELL.  The field
 * set must outlive the particle set. */
PG_API pg_status pg_pset_create(pg_fieldset *fs, int64_t n, const double *lon, const double *lat,
                         const double *depth, const double *time, double t0,
                         const uint64_t *ids, uint64_t id_base, int pos, uint64_t seed,
                         pg_pset **out);

/* Append particles between executes (the repeated releases of Sect. 3). */
PG_API pg_status pg_pset_add(pg_pset *ps, int64_t n, const double *lon, const double *lat,
                      const double *depth, const double *time, double t0, const uint64_t *ids,
                      uint64_t id_base);

/* Number of particles (alive and deleted) and of alive particles (the
 * ParticleSet of Sect. 2.1, whose particles deletion removes from the
 * computation, Sect. 3).  Either pointer may be NULL. */
PG_API pg_status pg_pset_size(const pg_pset *ps, int64_t *n, int64_t *n_alive);

/* Copy the particle state out (the particle variables of Sect. 2.1: lon,
 * lat, depth, time, plus id, step count and status), library order.  Any
 * pointer may be NULL.  Host or device destinations of n entries each,
 * positions widened to FP64. */
PG_API pg_status pg_pset_get(const pg_pset *ps, double *lon, double *lat, double *depth, double *time,
                      uint64_t *ids, uint32_t *steps, uint8_t *status, void *stream);

/* Particle variables (the extra Variables of the worked example's particle
 * class, Sect. 3): age[n] in seconds (0 at creation) and, for the sample
 * behaviour, vars[nvar * n] with variable j of particle i at vars[j * n + i]
 * (NaN until a step has sampled it); nvar is the number of scalar fields the
 * field set had when the particle set was created.  Library order, as
 * pg_pset_get; host or device destinations; either may be NULL. */
PG_API pg_status pg_pset_get_variables(const pg_pset *ps, double *age, double *vars, void *stream);

/* Tuning of the time loop (Sect. 2.2: the execution loop; not a paper
 * parameter): block size, re-sort interval and steps per launch.  Zero
 * fields take defaults; PG_ERR_ARG for a block that is not a multiple of 32
 * in [32, 1024] or negative intervals. */
PG_API pg_status pg_pset_set_tune(pg_pset *ps, const pg_tune *tune);

/* Advance every alive particle (the execute of Sect. 2.2 and 3): from the
 * particle set's time by `runtime` seconds with steps of dt (dt < 0 runs
 * backward in time).  Each particle steps while its own time lies before the
 * end time; the last step is shortened to land on it.  If output_dt > 0 and
 * out != NULL, `out` is called at every multiple of output_dt after the
 * start and at the end.  Writes the number of particle-steps taken to
 * *steps_done if non-NULL. */
PG_API pg_status pg_execute(pg_pset *ps, const pg_kernel *k, double runtime, double dt,
                     double output_dt, pg_output_cb out, void *user, void *stream,
                     int64_t *steps_done);

/* pg_execute with trajectory output in the ParticleFile's form (Sect. 3):
 * at every multiple of output_dt after the start and at the end, `rec` gets
 * the rows of that output time.  indexed = 0: every particle.  indexed = 1:
 * the 'indexed' format of Sect. 3, where particles are added and deleted
 * during the run: only the particles alive at that time and those deleted
 * since the previous output time (their last state and status), so each
 * particle's records end with its deletion.  The rows are packed on the GPU
 * and copied into a pinned two-slot ring on a side stream while the next
 * launch runs; `rec` for output k is called when output k + 1 has been
 * packed, and the last one before the call returns.  The ring holds 2 x
 * (41 + 8 nvar) bytes per particle of device and pinned host memory, kept by
 * the particle set for later executes. */
PG_API pg_status pg_execute_records(pg_pset *ps, const pg_kernel *k, double runtime, double dt,
                                    double output_dt, int indexed, pg_record_cb rec, void *user,
                                    void *stream, int64_t *steps_done);

/* Batched form: advance many releases (the repeated releases of Sect. 3),
 * each a particle set with its own kernel, dt (> 0) and runtime, over one
 * field set with all snapshots resident.  Every `window` seconds of
 * simulated time is one launch of a persistent kernel that walks a work list
 * of (release, tile) pairs, heaviest first.  Releases of at least 65,536
 * particles are Morton re-sorted before the first window and every
 * tune->resort_steps windows (0: never; in this call the field counts
 * windows, not steps; an interval of at least the number of windows sorts
 * before the first window only).  tune == NULL runs the autotuner: it times
 * each block size in {64, 128, 256} with each re-sort interval in {never, 1,
 * 2, 4, the whole run} over the first (up to) four windows (the sort before
 * the first window charged at the share of the run the trial covers, as it is
 * paid once) from a saved
 * copy of the state, restores the state and keeps the fastest; with
 * `tune_cache` (a file path, may be NULL) the choice is stored under a key of
 * the GPU name and the workload's shape and reused by later calls.  The
 * choice is written to *chosen if non-NULL.  use_graph != 0 captures the whole
 * window loop in one CUDA graph and launches it once.  Positions must be
 * PG_POS_F32.  Each release runs from its particle set's start time for its
 * runtime; particle-steps taken go to *steps_done. */
PG_API pg_status pg_execute_batch(int nrel, pg_pset *const *psets, const pg_kernel *const *kernels,
                                  const double *runtime, const double *dt, double window,
                                  const pg_tune *tune, pg_tune *chosen, const char *tune_cache,
                                  int use_graph, void *stream, int64_t *steps_done);

/* ------------------------------------------------- flow-map surrogate MLP */

/* A multilayer perceptron n_in -> width (x depth hidden layers, GELU) ->
 * n_out for the learned 24-hour flow map (not part of the paper's method; a
 * surrogate judged and backed by the RK4 of Sect. 2.1.1).  Weights are BF16
 * copies of FP32 master parameters; every matrix product runs on the tensor
 * cores with FP32 accumulation.  Widths are padded to multiples of 64 with
 * zeros.  He-uniform initialisation from `seed`. */
typedef struct pg_mlp pg_mlp;
PG_API pg_status pg_mlp_create(int n_in, int width, int depth, int n_out, uint64_t seed,
                               pg_mlp **out);
PG_API pg_status pg_mlp_destroy(pg_mlp *net);
/* Parameter counts: padded layout and the real (unpadded) network. */
PG_API pg_status pg_mlp_num_params(const pg_mlp *net, int64_t *padded, int64_t *real);
/* FP32 parameters in the padded layout, host memory: for each layer l, W_l
 * [dout x din] row-major then b_l [dout]; din/dout are the padded widths. */
PG_API pg_status pg_mlp_get_params(const pg_mlp *net, float *host);
PG_API pg_status pg_mlp_set_params(pg_mlp *net, const float *host);
/* Engine of the products: 0 warp-level mma.sync (default); 1 tcgen05 (5th-
 * generation tensor cores, accumulators in tensor memory): every product
 * whose widths are 64 or 256, and for the surrogate's shape (input and
 * output padded to 64, four hidden layers of 256) inference as one fused
 * kernel that keeps the activations on chip; 2 tcgen05 products without the
 * fused inference (layer by layer, for comparison). */
PG_API pg_status pg_mlp_set_engine(pg_mlp *net, int tcgen05);
/* y [M x n_out] = net(x [M x n_in]); device FP32 arrays, on `stream`. */
PG_API pg_status pg_mlp_forward(pg_mlp *net, const float *x, int64_t M, float *y, void *stream);
/* Gradient of L = 0.5 mean_rows sum_out (y - t)^2 for a batch (device x, t;
 * M a multiple of 32); loss to *loss, gradients (padded layout) to host
 * `grad` if non-NULL. */
PG_API pg_status pg_mlp_grad(pg_mlp *net, const float *x, const float *t, int64_t M, float *loss,
                             float *grad, void *stream);
/* One Adam step (beta 0.9, 0.999, eps 1e-8) on a batch. */
PG_API pg_status pg_mlp_train_step(pg_mlp *net, const float *x, const float *t, int64_t M,
                                   float lr, float *loss, void *stream);

/* Surrogate inputs of every particle of a set (FP32 positions on a resident
 * FP32 field set) at its current time, 37 floats per particle into device
 * x[n x 37]: the position inside its lon and lat cell (0..1), lat / 90,
 * depth / 1000 m, the phase of the field's period (0..1), then U and V
 * divided by 0.3 m/s at the 4 x 4 nodes i-1..i+2, j-1..j+2 around the cell,
 * interpolated linearly in depth and time to the particle.  Deleted
 * particles get zeros. */
PG_API pg_status pg_surrogate_features(const pg_pset *ps, float *x, void *stream);
/* Move every alive particle by y[n x 3] (device): cells of lon and lat and
 * units of 100 m of depth; time advances by `horizon` seconds.  Positions
 * leaving the domain delete the particle (status as for advection). */
PG_API pg_status pg_surrogate_apply(pg_pset *ps, const float *y, double horizon, void *stream);
/* Displacement of each particle from set a to set b (same particles in the
 * same order) in the units of pg_surrogate_apply, into device y[n x 3]. */
PG_API pg_status pg_pset_displacement(const pg_pset *a, const pg_pset *b, float *y, void *stream);

typedef struct {
    int64_t network_steps;      /* particle x network steps taken                     */
    int64_t checked;            /* particle checks where both kept the particle alive */
    int64_t rejected;           /* particles re-integrated with RK4                   */
    int64_t rk4_particle_steps; /* RK4 particle-steps spent on checks and fallback    */
    double error_sum;           /* sum of checked errors in cells                     */
    double seconds_network;     /* device time of the network steps                   */
    double seconds_rk4;         /* device time of checks and fallback                 */
    double seconds_total;       /* wall time of the call                              */
} pg_surrogate_stats;

/* Surrogate run: `nsteps` network steps of `horizon` seconds in blocks of
 * `check_every`.  The last step of every block is checked against RK4 with
 * steps of dt_check from the same state: particles whose position differs by
 * more than `threshold` cells (depth: layers), and particles that the network
 * or the checking RK4 deleted within the block, are re-integrated with RK4
 * from the start of the block (packed into a dense set, then written back);
 * all others take RK4's state for the checked step.  The kernel `k` is the
 * checking RK4's.  If the set's tuning has re-sorts (resort_steps > 0), the
 * particles are put in Morton order at the start of every block (their
 * storage order changes; ids are kept). */
PG_API pg_status pg_surrogate_run(pg_pset *ps, pg_mlp *net, const pg_kernel *k, int nsteps,
                                  int check_every, double horizon, double dt_check,
                                  double threshold, pg_surrogate_stats *stats, void *stream);

/* Morton re-sort now: order particles by the Morton code of their cell
 * indices and move deleted particles behind the alive ones. */
PG_API pg_status pg_pset_resort(pg_pset *ps, void *stream);

/* FP64 moments of the alive particles' positions (deleted ones excluded):
 * out[0..6] = count, sum lon, sum lat, sum depth, sum lon^2, sum lat^2,
 * sum depth^2, accumulated in FP64 in a fixed order (deterministic). */
PG_API pg_status pg_pset_moments(const pg_pset *ps, double out[7], void *stream);

/* FP64 moments of caller-owned particle arrays without allocating memory.
 * The paper has no counterpart: this call exists for callers that must not
 * allocate device memory while they run -- processes whose device memory
 * all belongs to their own allocator from start-up, and latency-critical
 * loops that cannot afford cudaMalloc/cudaFree round trips (cudaFree also
 * synchronises the whole device).  It sums as pg_pset_moments does (count,
 * sums and sums of squares of lon, lat, depth over particles whose status is
 * 0), over device arrays lon[n], lat[n], depth[n] (NULL: zeros) and
 * status[n] (NULL: all alive), and writes the 7 doubles to the device
 * pointer `out`, asynchronously on `stream`.
 *   - No allocation: the partial sums live in a fixed device array of the
 *     library (229,376 bytes, held on every GPU that loads the library until
 *     the process exits).  n may be at most 268,435,456; larger n returns
 *     PG_ERR_ARG before any work.
 *   - The first call on a device looks up that array's device address
 *     (cudaGetSymbolAddress) with the device current; make that first call
 *     before any stream capture.  With CUDA's lazy module loading (the
 *     default) that first call is also when the array is placed in device
 *     memory, so make it before the caller's own allocator reserves the
 *     device's memory, or run with CUDA_MODULE_LOADING=EAGER.
 *   - The looked-up address is kept for the life of the process: the call
 *     does not survive cudaDeviceReset (nor does any other object of this
 *     library).
 *   - Every call shares the array and leaves the last call's partial sums in
 *     it (each call overwrites all it reads, so nothing needs clearing).
 *     Calls whose work overlaps on the GPU, on any streams, race on it:
 *     order them on one stream or synchronise between them.
 *   - Errors: PG_ERR_ARG (NULL pointers, n out of range), PG_ERR_CUDA. */
PG_API pg_status pg_moments_f64_noalloc(const double *lon, const double *lat,
                                        const double *depth, const uint8_t *status, int64_t n,
                                        double *out, void *stream);

/* Checkpoint: write / read the complete particle state (positions, times,
 * ids, step counters, status, age and sampled variables, seed) to a file, so
 * that a run executed in a loop of pg_execute calls (Sect. 3) can stop and
 * resume.  Restoring gives a set that continues bit-identically; the field
 * set must have as many scalar fields as the saved set had variables
 * (PG_ERR_ARG otherwise, and for a file that is not a checkpoint). */
PG_API pg_status pg_pset_save(const pg_pset *ps, const char *path);
PG_API pg_status pg_pset_restore(pg_fieldset *fs, const char *path, pg_pset **out);

PG_API pg_status pg_pset_destroy(pg_pset *ps);

/* ------------------------------------------------------- instrumentation */

/* CUDA-event timing of the advection launches of pg_execute, recorded on the
 * execute's stream around every launch.  Returns the time and number of
 * launches accumulated since timing was last enabled; enable = 1 turns timing
 * on and resets the totals, 0 turns it off and resets, -1 only reads. */
PG_API pg_status pg_pset_kernel_timing(pg_pset *ps, int enable, double *total_ms,
                                       int64_t *launches);

/* Streaming statistics of a field set: snapshot uploads and the bytes copied
 * host-to-device for them since the last reset (reset != 0 clears after
 * reading). */
PG_API pg_status pg_fieldset_stats(pg_fieldset *fs, int reset, int64_t *uploads,
                                   int64_t *h2d_bytes);

/* Measured read bandwidth of the L2 cache in GB/s (the bound of a gather
 * that hits in L2; the paper names field sampling as the dominant cost,
 * Sect. 2.3, 5.1): a device buffer of `bytes` (at least 1 MiB, a multiple of
 * 16, at most half the L2) is filled, read once to warm the cache, then read
 * 16 times per launch with coalesced 16-byte loads that bypass L1; the best
 * of `reps` launches timed with CUDA events on `stream` goes to *gbs.  The
 * buffer is allocated and freed by the call. */
PG_API pg_status pg_measure_l2_read(size_t bytes, int reps, double *gbs, void *stream);

/* Number of kernel launches the library has made in this process. */
PG_API pg_status pg_launch_count(int64_t *count);

/* ------------------------------------------------------------ test hooks */

/* Make every later device allocation of the library fail once the library
 * has allocated `bytes` more than it holds now (negative: no limit).  Used to
 * test that a failed allocation leaves objects unchanged. */
PG_API pg_status pg_debug_set_alloc_limit(int64_t bytes);

/* Run the bounded mbarrier wait of the tcgen05 kernels (the MLP products and
 * the fused inference) on a barrier phase that nothing completes, with no
 * copy or product in flight: the wait gives up after `polls` polls (1 to
 * 1e7), the kernel records it and the call returns PG_ERR_TIMEOUT, as those
 * kernels report a product or copy that never signals; the context stays
 * usable.  Used to test the failure path without faulting the GPU. */
PG_API pg_status pg_debug_bounded_wait(int64_t polls, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* PARCELS_GB_H */
