/*
 * parcels_oracle.c -- plain, slow FP64 CPU oracle of the particle-advection step.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load this library.  The product path
 * (the CUDA library) shares no code, header or constant table with this file.
 *
 * What it computes (Lange & van Sebille, "Parcels v0.9", arXiv 1707.05163):
 *   - Eq. 1: X(t+dt) = X(t) + integral of v(x, tau) over [t, t+dt] + dX_b,
 *     time-stepped with classical RK4 (Sect. 2.1.1) or Euler-forward;
 *   - velocities interpolated linearly in space (bi/trilinear) and linearly
 *     in time on a rectilinear grid whose axes depend on one coordinate each
 *     (Sect. 2.3 and 2.4);
 *   - on a spherical mesh, m/s are turned into degrees/s (Sect. 4.2.2);
 *   - behaviours composed after advection: Brownian motion with uniform K_h and
 *     normal variates (Sect. 2.1.2, 4.2.7), constant sinking (Eq. 1's dX_b);
 *   - out-of-bounds recovery = delete the particle (Sect. 2.1.2, 3).
 * Readings where the paper is silent (all stated in the design notes):
 *   - RK4 stage times t, t+dt/2, t+dt/2, t+dt; X += (k1+2k2+2k3+k4)/6*dt;
 *   - the bilinear/trilinear/time weights are evaluated in the order written in
 *     interp_2d / sample_fields below;
 *   - cell tie-break: i is the largest index with x_i <= p, capped at n-2;
 *   - periodic zonal boundary: the grid spans 360 deg minus one cell, the wrap
 *     cell joins node n-1 to node 0, positions are reduced modulo 360 into
 *     [x_0, x_0+360);
 *   - metres per degree D = 1852*60 (one nautical mile per arc-minute), taken at
 *     the latitude of the position being evaluated;
 *   - random numbers: Philox4x32-10 (Salmon et al., SC'11) keyed by the seed,
 *     counter (id lo, id hi, step, stream), then Box-Muller;
 *   - a step whose stage or final position leaves the domain is not applied and
 *     the particle is deleted (status != 0);
 *   - nearest-neighbour interpolation (Sect. 2.3) picks, on each axis, the
 *     node nearest to the position, the lower one on a tie; time stays linear;
 *   - the worked example of Sect. 3 (sinking phase, age with a maximum, sampled
 *     temperature, constants carried by the FieldSet) as three behaviours that
 *     run after advection, Brownian motion and sinking, in this order:
 *       settle: while the depth differs from the dwelling depth at the step's
 *         start, the depth moves by w_sink * h and stops at the dwelling depth
 *         when it reaches or passes it; a particle that starts the step at the
 *         dwelling depth holds it (vertical advection and sinking discarded);
 *       age: age += |h| for every step (with settle: every step that starts at
 *         the dwelling depth); once age >= max_age the particle is deleted with
 *         status 4 and keeps the step's result;
 *       sample: each scalar field is interpolated at the step's new position
 *         and time into the particle's variable (NaN where the field is NaN);
 *   - adaptive RKF45 (Sect. 2.1.1 names Runge-Kutta-Fehlberg): the Fehlberg
 *     4(5) pair; a trial step of length h gives the fourth-order X4 and the
 *     fifth-order X5; its error is the largest of |X5 - X4| over the axes in
 *     metres (degrees times metres per degree on a sphere, at the latitude of
 *     X4); the trial is accepted when the error is at most the tolerance or
 *     |h| is at the minimum step, and the particle moves to X4; a rejected
 *     trial halves the particle's step length (not below the minimum) and is
 *     repeated from the same state; after an accepted step whose error is
 *     below a tenth of the tolerance, taken at the particle's full step
 *     length, that length doubles (not above the maximum).  Each particle
 *     keeps its step length between steps and executes; a step is shortened
 *     to land on the stop time (the next output time) and on the end time.
 * Philox4x32-10 is pinned by the generator's published known-answer vectors;
 * the word-to-uniform mapping of Box-Muller by a value computed by hand from
 * one of them.
 *
 * Compiled with -ffp-contract=off so no multiply-add is fused behind our back.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* Public structures (mirrored by ctypes in oracle.py).                      */
/* ------------------------------------------------------------------------ */
typedef struct {
    int nx, ny, nz;               /* nz == 1: two-dimensional field            */
    const double *lon, *lat, *depth;
    int mesh;                     /* 0: flat, metres; 1: spherical, degrees    */
    int periodic_lon;             /* zonal wrap (spherical global grids)       */
    int nfields;                  /* 2: U,V   3: U,V,W                         */
    int nt;                       /* number of snapshots; 1 = steady           */
    const double *times;          /* [nt], strictly increasing                 */
    double period;                /* > 0: field repeats with this period       */
    int dtype;                    /* 0: double data, 1: float data             */
    const void *data;             /* [nt][nfields][nz][ny][nx], lon fastest    */
    double deg_m;                 /* metres per degree on the sphere           */
    int interp;                   /* velocities: 0 linear, 1 nearest node      */
    int ntracers;                 /* scalar fields sampled into variables      */
    const void *tracer[2];        /* each [nt][nz][ny][nx], dtype as data      */
    int tracer_interp[2];         /* 0 linear, 1 nearest node                  */
} or_fieldset;

typedef struct {
    int scheme;                   /* 0: Euler-forward, 1: RK4                  */
    unsigned behaviours;          /* bit 0: Brownian, bit 1: sinking           */
    double kh;                    /* m^2/s                                     */
    double w_sink;                /* m/s, positive downward                    */
    uint64_t seed;
    double dwell_depth;           /* settle: depth where the vertical move ends */
    double max_age;               /* age: deletion age in seconds              */
    double rk45_tol;              /* RKF45: error tolerance per step, metres   */
    double rk45_hmin, rk45_hmax;  /* RKF45: smallest and largest step, seconds */
} or_kernel;

enum { OR_ALIVE = 0, OR_OOB_HORIZ = 1, OR_OOB_DEPTH = 2, OR_NAN = 3, OR_DELETED = 4 };
enum { OR_BROWNIAN = 1u, OR_SINK = 2u, OR_SETTLE = 4u, OR_AGE = 8u, OR_SAMPLE = 16u };

/* ------------------------------------------------------------------------ */
/* Cell search (Sect. 2.4: rectilinear axes).                                */
/* ------------------------------------------------------------------------ */

/* Locate p on the increasing axis x[0..n-1].  Returns 0 and (i, xi) with
 * x[i] <= p, p <= x[i+1], xi = (p - x[i]) / (x[i+1] - x[i]); i is the largest
 * such index but at most n-2.  Returns 1 when p is outside [x0, x_{n-1}] or NaN.
 * A single-node axis always gives i = 0, xi = 0. */
int or_locate(const double *x, int n, double p, int *i, double *xi)
{
    if (!(p >= x[0] && p <= x[n - 1])) return 1;
    if (n == 1) { *i = 0; *xi = 0.0; return 0; }
    int lo = 0, hi = n - 1;            /* x[lo] <= p, and p < x[hi] or hi == n-1 */
    while (hi - lo > 1) {
        int mid = lo + (hi - lo) / 2;
        if (x[mid] <= p) lo = mid; else hi = mid;
    }
    *i = lo;
    *xi = (p - x[lo]) / (x[lo + 1] - x[lo]);
    return 0;
}

/* Reduce a longitude into [x0, x0 + 360). */
double or_wrap_lon(double p, double x0)
{
    double q = fmod(p - x0, 360.0);
    if (q < 0.0) q += 360.0;
    if (q >= 360.0) q -= 360.0;
    return x0 + q;
}

/* Zonal search.  On a periodic axis, the position is wrapped first; a point
 * past the last node falls in the wrap cell (n-1 -> 0) whose far edge is
 * x0 + 360.  Returns the two corner indices and the fraction. */
int or_locate_lon(const double *x, int n, int periodic, double p,
                  int *i0, int *i1, double *xi)
{
    if (!periodic) {
        int r = or_locate(x, n, p, i0, xi);
        if (r) return r;
        *i1 = (n == 1) ? *i0 : *i0 + 1;
        return 0;
    }
    if (!isfinite(p)) return 1;
    double q = or_wrap_lon(p, x[0]);
    if (q >= x[n - 1]) {
        *i0 = n - 1;
        *i1 = 0;
        *xi = (q - x[n - 1]) / ((x[0] + 360.0) - x[n - 1]);
        return 0;
    }
    int r = or_locate(x, n, q, i0, xi);
    *i1 = *i0 + 1;
    return r;
}

/* ------------------------------------------------------------------------ */
/* Time interval (Sect. 2.4: linear in time between two snapshots).          */
/* ------------------------------------------------------------------------ */

/* Find the snapshots s0, s1 bracketing t and the fraction tau.  A steady field
 * (nt == 1) gives s0 = s1 = 0, tau = 0.  A periodic field reduces t into
 * [t0, t0 + period); past the last snapshot it interpolates towards snapshot
 * 0 at t0 + period.  Returns 1 for t outside a non-periodic time range. */
int or_time_interval(const or_fieldset *fs, double t, int *s0, int *s1, double *tau)
{
    const double *T = fs->times;
    int nt = fs->nt;
    if (nt == 1) { *s0 = 0; *s1 = 0; *tau = 0.0; return 0; }
    double tt = t;
    if (fs->period > 0.0) {
        tt = fmod(t - T[0], fs->period);
        if (tt < 0.0) tt += fs->period;
        tt = T[0] + tt;
        if (tt >= T[nt - 1]) {
            *s0 = nt - 1;
            *s1 = 0;
            *tau = (tt - T[nt - 1]) / ((T[0] + fs->period) - T[nt - 1]);
            return 0;
        }
    }
    int s;
    double f;
    if (or_locate(T, nt, tt, &s, &f)) return 1;
    *s0 = s;
    *s1 = s + 1;
    *tau = f;
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Interpolation.                                                            */
/* ------------------------------------------------------------------------ */

static double field_value(const or_fieldset *fs, int s, int f, int k, int j, int i)
{
    size_t idx = ((((size_t)s * fs->nfields + f) * fs->nz + k) * fs->ny + j) * fs->nx + i;
    if (fs->dtype == 0) return ((const double *)fs->data)[idx];
    return (double)((const float *)fs->data)[idx];
}

static double tracer_value(const or_fieldset *fs, int tr, int s, int k, int j, int i)
{
    size_t idx = (((size_t)s * fs->nz + k) * fs->ny + j) * fs->nx + i;
    if (fs->dtype == 0) return ((const double *)fs->tracer[tr])[idx];
    return (double)((const float *)fs->tracer[tr])[idx];
}

/* Nearest node of a cell on one axis: the lower node unless the fraction is
 * above one half (a tie goes to the lower node). */
static int nearest_node(int lo, int hi, double frac)
{
    return frac <= 0.5 ? lo : hi;
}

/* Bilinear weights applied as (w00 f00 + w10 f10) + (w11 f11 + w01 f01). */
static double interp_2d(const or_fieldset *fs, int s, int f, int k,
                        int i0, int i1, int j0, int j1, double xi, double eta)
{
    double f00 = field_value(fs, s, f, k, j0, i0);
    double f10 = field_value(fs, s, f, k, j0, i1);
    double f01 = field_value(fs, s, f, k, j1, i0);
    double f11 = field_value(fs, s, f, k, j1, i1);
    double w00 = (1.0 - xi) * (1.0 - eta);
    double w10 = xi * (1.0 - eta);
    double w11 = xi * eta;
    double w01 = (1.0 - xi) * eta;
    return (w00 * f00 + w10 * f10) + (w11 * f11 + w01 * f01);
}

/* Trilinear = linear in zeta between the bilinear values of levels k, k+1. */
static double interp_space(const or_fieldset *fs, int s, int f, int i0, int i1,
                           int j0, int j1, int k0, int k1, double xi, double eta,
                           double zeta)
{
    double a = interp_2d(fs, s, f, k0, i0, i1, j0, j1, xi, eta);
    if (fs->nz == 1) return a;
    double b = interp_2d(fs, s, f, k1, i0, i1, j0, j1, xi, eta);
    return (1.0 - zeta) * a + zeta * b;
}

/* Sample the raw fields (U, V[, W] in m/s) at a position and time.
 * Returns 0 or an OR_* status: horizontal/depth out of bounds, NaN sample.
 * Time outside a non-periodic range returns -1. */
int or_sample(const or_fieldset *fs, double t, double lon, double lat, double depth,
              double *out)
{
    int i0, i1, j0, j1, k0 = 0, k1 = 0;
    double xi, eta, zeta = 0.0;
    if (or_locate_lon(fs->lon, fs->nx, fs->periodic_lon, lon, &i0, &i1, &xi)) return OR_OOB_HORIZ;
    if (or_locate(fs->lat, fs->ny, lat, &j0, &eta)) return OR_OOB_HORIZ;
    j1 = (fs->ny == 1) ? j0 : j0 + 1;
    if (fs->nz > 1) {
        if (or_locate(fs->depth, fs->nz, depth, &k0, &zeta)) return OR_OOB_DEPTH;
        k1 = k0 + 1;
    }
    int s0, s1;
    double tau;
    if (or_time_interval(fs, t, &s0, &s1, &tau)) return -1;
    int in = nearest_node(i0, i1, xi), jn = nearest_node(j0, j1, eta);
    int kn = nearest_node(k0, k1, zeta);
    for (int f = 0; f < fs->nfields; ++f) {
        double a, v;
        if (fs->interp == 1) a = field_value(fs, s0, f, kn, jn, in);
        else a = interp_space(fs, s0, f, i0, i1, j0, j1, k0, k1, xi, eta, zeta);
        v = a;
        if (fs->nt > 1) {
            double b;
            if (fs->interp == 1) b = field_value(fs, s1, f, kn, jn, in);
            else b = interp_space(fs, s1, f, i0, i1, j0, j1, k0, k1, xi, eta, zeta);
            v = a + (b - a) * tau;
        }
        if (!(v == v)) return OR_NAN;
        out[f] = v;
    }
    if (fs->nfields == 2) out[2] = 0.0;
    return OR_ALIVE;
}

/* Sample scalar field tr (Sect. 3: a field sampled by a kernel) at a
 * position and time, linearly or at the nearest node in space as the field
 * says, linearly in time.  Returns 0 and the value (NaN where the field is
 * NaN), an OR_OOB_* status, or -1 for a time outside a non-periodic range. */
int or_sample_tracer(const or_fieldset *fs, int tr, double t, double lon, double lat,
                     double depth, double *out)
{
    int i0, i1, j0, j1, k0 = 0, k1 = 0;
    double xi, eta, zeta = 0.0;
    if (or_locate_lon(fs->lon, fs->nx, fs->periodic_lon, lon, &i0, &i1, &xi)) return OR_OOB_HORIZ;
    if (or_locate(fs->lat, fs->ny, lat, &j0, &eta)) return OR_OOB_HORIZ;
    j1 = (fs->ny == 1) ? j0 : j0 + 1;
    if (fs->nz > 1) {
        if (or_locate(fs->depth, fs->nz, depth, &k0, &zeta)) return OR_OOB_DEPTH;
        k1 = k0 + 1;
    }
    int s0, s1;
    double tau;
    if (or_time_interval(fs, t, &s0, &s1, &tau)) return -1;
    double val[2];
    for (int q = 0; q < (fs->nt > 1 ? 2 : 1); ++q) {
        int s = q == 0 ? s0 : s1;
        if (fs->tracer_interp[tr] == 1) {
            val[q] = tracer_value(fs, tr, s, nearest_node(k0, k1, zeta), nearest_node(j0, j1, eta),
                                  nearest_node(i0, i1, xi));
        } else {
            double w00 = (1.0 - xi) * (1.0 - eta);
            double w10 = xi * (1.0 - eta);
            double w11 = xi * eta;
            double w01 = (1.0 - xi) * eta;
            double a = (w00 * tracer_value(fs, tr, s, k0, j0, i0) + w10 * tracer_value(fs, tr, s, k0, j0, i1)) +
                       (w11 * tracer_value(fs, tr, s, k0, j1, i1) + w01 * tracer_value(fs, tr, s, k0, j1, i0));
            if (fs->nz > 1) {
                double b = (w00 * tracer_value(fs, tr, s, k1, j0, i0) + w10 * tracer_value(fs, tr, s, k1, j0, i1)) +
                           (w11 * tracer_value(fs, tr, s, k1, j1, i1) + w01 * tracer_value(fs, tr, s, k1, j1, i0));
                a = (1.0 - zeta) * a + zeta * b;
            }
            val[q] = a;
        }
    }
    *out = fs->nt > 1 ? val[0] + (val[1] - val[0]) * tau : val[0];
    return OR_ALIVE;
}

/* Velocity in position units per second: m/s on a flat mesh; on a sphere
 * u / (D cos(lat)) and v / D degrees per second; W stays in m/s. */
int or_velocity(const or_fieldset *fs, double t, double lon, double lat, double depth,
                double *vel)
{
    int r = or_sample(fs, t, lon, lat, depth, vel);
    if (r) return r;
    if (fs->mesh == 1) {
        const double deg2rad = 3.14159265358979323846 / 180.0;
        vel[0] = vel[0] / (fs->deg_m * cos(lat * deg2rad));
        vel[1] = vel[1] / fs->deg_m;
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) and Box-Muller.         */
/* ------------------------------------------------------------------------ */

/* Ten rounds; each round multiplies words 0 and 2 by the two Philox
 * multipliers and mixes the high halves with words 1, 3 and the round key;
 * the key advances by the two Weyl constants between rounds. */
void or_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int r = 0; r < 10; ++r) {
        if (r > 0) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
        uint64_t p0 = (uint64_t)0xD2511F53u * c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Two standard normal variates for (seed, particle id, step).  Words 0,1 form
 * a 53-bit uniform u1 in (0, 1], words 2,3 a 53-bit uniform u2 in [0, 1);
 * n1 = sqrt(-2 ln u1) cos(2 pi u2), n2 = sqrt(-2 ln u1) sin(2 pi u2). */
void or_normal_pair(uint64_t seed, uint64_t id, uint32_t step, double *n1, double *n2)
{
    uint32_t ctr[4] = {(uint32_t)id, (uint32_t)(id >> 32), step, 0u};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t r[4];
    or_philox4x32_10(ctr, key, r);
    uint64_t m1 = ((uint64_t)(r[0] >> 5) << 26) | (uint64_t)(r[1] >> 6);
    uint64_t m2 = ((uint64_t)(r[2] >> 5) << 26) | (uint64_t)(r[3] >> 6);
    double u1 = ((double)m1 + 1.0) * (1.0 / 9007199254740992.0);
    double u2 = (double)m2 * (1.0 / 9007199254740992.0);
    double rad = sqrt(-2.0 * log(u1));
    double ang = 6.283185307179586 * u2;
    *n1 = rad * cos(ang);
    *n2 = rad * sin(ang);
}

/* ------------------------------------------------------------------------ */
/* One step of Eq. 1 for one particle.                                       */
/* ------------------------------------------------------------------------ */

static int out_of_domain(const or_fieldset *fs, double lon, double lat, double depth)
{
    if (!fs->periodic_lon && !(lon >= fs->lon[0] && lon <= fs->lon[fs->nx - 1])) return OR_OOB_HORIZ;
    if (fs->periodic_lon && !(lon == lon)) return OR_OOB_HORIZ;   /* no longer a number */
    if (!(lat >= fs->lat[0] && lat <= fs->lat[fs->ny - 1])) return OR_OOB_HORIZ;
    if (fs->nz > 1 && !(depth >= fs->depth[0] && depth <= fs->depth[fs->nz - 1])) return OR_OOB_DEPTH;
    return OR_ALIVE;
}

/* Advance one particle by h seconds.  On success the new state is written and
 * 0 returned (OR_DELETED when the age behaviour deleted it, with the new state
 * written); otherwise the state is left untouched and the status returned.
 * age and vars (stride vstride between variables) are written on success. */
static int finish_step(const or_fieldset *fs, const or_kernel *kn, double *plon, double *plat,
                       double *pdep, double t, double h, uint64_t id, uint32_t step,
                       double *page, double *pvars, int64_t vstride,
                       double nlon, double nlat, double ndep);

/* The Fehlberg 4(5) pair: stage times c, stage weights a (row i uses stages
 * 0..i-1), fourth- and fifth-order weights b4, b5. */
static const double RKF_C[6] = {0.0, 1.0 / 4.0, 3.0 / 8.0, 12.0 / 13.0, 1.0, 1.0 / 2.0};
static const double RKF_A[6][5] = {
    {0, 0, 0, 0, 0},
    {1.0 / 4.0, 0, 0, 0, 0},
    {3.0 / 32.0, 9.0 / 32.0, 0, 0, 0},
    {1932.0 / 2197.0, -7200.0 / 2197.0, 7296.0 / 2197.0, 0, 0},
    {439.0 / 216.0, -8.0, 3680.0 / 513.0, -845.0 / 4104.0, 0},
    {-8.0 / 27.0, 2.0, -3544.0 / 2565.0, 1859.0 / 4104.0, -11.0 / 40.0}};
static const double RKF_B4[6] = {25.0 / 216.0, 0.0, 1408.0 / 2565.0, 2197.0 / 4104.0, -1.0 / 5.0, 0.0};
static const double RKF_B5[6] = {16.0 / 135.0, 0.0, 6656.0 / 12825.0, 28561.0 / 56430.0,
                                 -9.0 / 50.0, 2.0 / 55.0};

/* One RKF45 trial of length h from (lon, lat, dep) at t: the fourth-order
 * position in out4 and the error estimate in metres.  Returns 0 or the
 * status of a stage (out of the domain, NaN velocity). */
int or_rkf45_trial(const or_fieldset *fs, double lon, double lat, double dep, double t,
                   double h, double *out4, double *err_m)
{
    double k[6][3];
    for (int i = 0; i < 6; ++i) {
        double px = lon, py = lat, pz = dep;
        for (int j = 0; j < i; ++j) {
            px = px + h * RKF_A[i][j] * k[j][0];
            py = py + h * RKF_A[i][j] * k[j][1];
            pz = pz + h * RKF_A[i][j] * k[j][2];
        }
        int r = or_velocity(fs, t + RKF_C[i] * h, px, py, pz, k[i]);
        if (r) return r;
    }
    double d4[3] = {0, 0, 0}, d5[3] = {0, 0, 0};
    for (int i = 0; i < 6; ++i)
        for (int q = 0; q < 3; ++q) {
            d4[q] = d4[q] + RKF_B4[i] * k[i][q];
            d5[q] = d5[q] + RKF_B5[i] * k[i][q];
        }
    out4[0] = lon + h * d4[0];
    out4[1] = lat + h * d4[1];
    out4[2] = dep + h * d4[2];
    double ex = fabs(h * (d5[0] - d4[0])), ey = fabs(h * (d5[1] - d4[1]));
    double ez = fabs(h * (d5[2] - d4[2]));
    if (fs->mesh == 1) {
        const double deg2rad = 3.14159265358979323846 / 180.0;
        ex = ex * fs->deg_m * cos(out4[1] * deg2rad);
        ey = ey * fs->deg_m;
    }
    double e = ex > ey ? ex : ey;
    *err_m = e > ez ? e : ez;
    return 0;
}

static int step_one(const or_fieldset *fs, const or_kernel *kn, double *plon, double *plat,
                    double *pdep, double t, double h, uint64_t id, uint32_t step,
                    double *page, double *pvars, int64_t vstride)
{
    double lon = *plon, lat = *plat, dep = *pdep;
    double k1[3], k2[3], k3[3], k4[3];
    double nlon, nlat, ndep;
    int r;
    if (kn->scheme == 0) {
        if ((r = or_velocity(fs, t, lon, lat, dep, k1))) return r;
        nlon = lon + k1[0] * h;
        nlat = lat + k1[1] * h;
        ndep = dep + k1[2] * h;
    } else {
        double half = 0.5 * h;
        if ((r = or_velocity(fs, t, lon, lat, dep, k1))) return r;
        if ((r = or_velocity(fs, t + half, lon + k1[0] * half, lat + k1[1] * half,
                             dep + k1[2] * half, k2))) return r;
        if ((r = or_velocity(fs, t + half, lon + k2[0] * half, lat + k2[1] * half,
                             dep + k2[2] * half, k3))) return r;
        if ((r = or_velocity(fs, t + h, lon + k3[0] * h, lat + k3[1] * h,
                             dep + k3[2] * h, k4))) return r;
        nlon = lon + (k1[0] + 2.0 * k2[0] + 2.0 * k3[0] + k4[0]) / 6.0 * h;
        nlat = lat + (k1[1] + 2.0 * k2[1] + 2.0 * k3[1] + k4[1]) / 6.0 * h;
        ndep = dep + (k1[2] + 2.0 * k2[2] + 2.0 * k3[2] + k4[2]) / 6.0 * h;
    }
    return finish_step(fs, kn, plon, plat, pdep, t, h, id, step, page, pvars, vstride,
                       nlon, nlat, ndep);
}

/* The part of a step after advection: behaviours, the zonal wrap, the
 * domain test, and on success the new state, age and sampled variables. */
static int finish_step(const or_fieldset *fs, const or_kernel *kn, double *plon, double *plat,
                       double *pdep, double t, double h, uint64_t id, uint32_t step,
                       double *page, double *pvars, int64_t vstride,
                       double nlon, double nlat, double ndep)
{
    double dep = *pdep;
    int r;
    if (kn->behaviours & OR_BROWNIAN) {
        double n1, n2;
        or_normal_pair(kn->seed, id, step, &n1, &n2);
        double sigma = sqrt(2.0 * kn->kh * fabs(h));
        double dx = sigma * n1, dy = sigma * n2;
        if (fs->mesh == 1) {
            const double deg2rad = 3.14159265358979323846 / 180.0;
            dx = dx / (fs->deg_m * cos(nlat * deg2rad));
            dy = dy / fs->deg_m;
        }
        nlon = nlon + dx;
        nlat = nlat + dy;
    }
    if (kn->behaviours & OR_SINK) ndep = ndep + kn->w_sink * h;
    int dwelling = 0;                    /* the step starts at the dwelling depth */
    if (kn->behaviours & OR_SETTLE) {
        if (dep == kn->dwell_depth) {
            dwelling = 1;
            ndep = kn->dwell_depth;
        } else {
            double moved = ndep + kn->w_sink * h;
            if ((dep - kn->dwell_depth) * (moved - kn->dwell_depth) <= 0.0) moved = kn->dwell_depth;
            ndep = moved;
        }
    }
    if (fs->periodic_lon) nlon = or_wrap_lon(nlon, fs->lon[0]);
    if ((r = out_of_domain(fs, nlon, nlat, ndep))) return r;
    *plon = nlon; *plat = nlat; *pdep = ndep;
    int status = OR_ALIVE;
    if (kn->behaviours & OR_AGE) {
        if (!(kn->behaviours & OR_SETTLE) || dwelling) *page = *page + fabs(h);
        if (*page >= kn->max_age) status = OR_DELETED;
    }
    if (kn->behaviours & OR_SAMPLE) {
        for (int q = 0; q < fs->ntracers; ++q) {
            double v;
            if (or_sample_tracer(fs, q, t + h, nlon, nlat, ndep, &v) == OR_ALIVE)
                pvars[q * vstride] = v;
        }
    }
    return status;
}

/* ------------------------------------------------------------------------ */
/* Driver: many particles, threads over particle ranges.                     */
/* ------------------------------------------------------------------------ */

typedef struct {
    const or_fieldset *fs;
    const or_kernel *kn;
    double *lon, *lat, *depth, *time;
    const uint64_t *id;
    uint32_t *step;
    uint8_t *status;
    double *age, *vars;            /* age[n], vars[ntracers][n]; may be NULL */
    double *hstep;                 /* RKF45 step lengths [n]; may be NULL      */
    int64_t n;
    double dt, t_stop, t_end;
    int64_t begin, end;
    int64_t steps_done;
} or_job;

/* RKF45 steps of particle p from time *pt while its time lies before t_stop
 * and t_end; returns the steps taken. */
static int64_t run_rkf45(or_job *jb, int64_t p, double *pt)
{
    const or_kernel *kn = jb->kn;
    double sgn = jb->dt > 0.0 ? 1.0 : -1.0;
    double t = *pt;
    double hp = jb->hstep ? jb->hstep[p] : 0.0;
    if (!(sgn * hp > 0.0)) hp = jb->dt;
    int64_t done = 0;
    double target = sgn * (jb->t_stop - jb->t_end) < 0.0 ? jb->t_stop : jb->t_end;
    while (sgn * (jb->t_stop - t) > 0.0 && sgn * (jb->t_end - t) > 0.0) {
        double h = hp;
        int clipped = 0;
        if (sgn * (target - t) < sgn * h) { h = target - t; clipped = 1; }
        double x4[3], err;
        int r = or_rkf45_trial(jb->fs, jb->lon[p], jb->lat[p], jb->depth[p], t, h, x4, &err);
        if (r) { jb->status[p] = (uint8_t)r; break; }
        if (err > kn->rk45_tol && fabs(h) > kn->rk45_hmin) {
            double nh = fabs(h) / 2.0;
            if (nh < kn->rk45_hmin) nh = kn->rk45_hmin;
            hp = sgn * nh;
            continue;
        }
        double age_dummy = 0.0;
        r = finish_step(jb->fs, kn, &jb->lon[p], &jb->lat[p], &jb->depth[p], t, h, jb->id[p],
                        jb->step[p], jb->age ? &jb->age[p] : &age_dummy,
                        jb->vars ? &jb->vars[p] : NULL, jb->n, x4[0], x4[1], x4[2]);
        if (r && r != OR_DELETED) { jb->status[p] = (uint8_t)r; break; }
        t = t + h;
        jb->step[p] += 1u;
        ++done;
        if (!clipped && err < kn->rk45_tol / 10.0) {
            double nh = 2.0 * fabs(hp);
            if (nh > kn->rk45_hmax) nh = kn->rk45_hmax;
            hp = sgn * nh;
        }
        if (r == OR_DELETED) { jb->status[p] = (uint8_t)r; break; }
    }
    if (jb->hstep) jb->hstep[p] = hp;
    *pt = t;
    return done;
}

/* A particle steps while its time lies before t_stop and before t_end (in the
 * direction of dt); the step length is dt, shortened only to land on t_end. */
static void *run_range(void *arg)
{
    or_job *jb = (or_job *)arg;
    double sgn = jb->dt > 0.0 ? 1.0 : -1.0;
    int64_t done = 0;
    for (int64_t p = jb->begin; p < jb->end; ++p) {
        if (jb->status[p] != OR_ALIVE) continue;
        double t = jb->time[p];
        if (jb->kn->scheme == 2) {
            done += run_rkf45(jb, p, &t);
            jb->time[p] = t;
            continue;
        }
        while (sgn * (jb->t_stop - t) > 0.0 && sgn * (jb->t_end - t) > 0.0) {
            double h = jb->dt;
            if (sgn * (jb->t_end - t) < sgn * h) h = jb->t_end - t;
            double age_dummy = 0.0;
            int r = step_one(jb->fs, jb->kn, &jb->lon[p], &jb->lat[p], &jb->depth[p],
                             t, h, jb->id[p], jb->step[p], jb->age ? &jb->age[p] : &age_dummy,
                             jb->vars ? &jb->vars[p] : NULL, jb->n);
            if (r == OR_DELETED) {          /* the step was taken, then the age deleted it */
                t = t + h;
                jb->step[p] += 1u;
                ++done;
                jb->status[p] = (uint8_t)r;
                break;
            }
            if (r) { jb->status[p] = (uint8_t)r; break; }
            t = t + h;
            jb->step[p] += 1u;
            ++done;
        }
        jb->time[p] = t;
    }
    jb->steps_done = done;
    return NULL;
}

/* Advance n particles.  Returns the number of particle-steps taken, or -1 if
 * the time span leaves a non-periodic field's time range. */
int64_t or_run(const or_fieldset *fs, const or_kernel *kn, int64_t n, double *lon,
               double *lat, double *depth, double *time, const uint64_t *id,
               uint32_t *step, uint8_t *status, double *age, double *vars, double *hstep,
               double dt, double t_stop, double t_end, int nthreads)
{
    if (n <= 0) return 0;
    if ((kn->behaviours & OR_SAMPLE) && fs->ntracers > 0 && !vars) return -2;
    if (fs->nt > 1 && fs->period <= 0.0) {
        for (int64_t p = 0; p < n; ++p) {
            if (status[p] != OR_ALIVE) continue;
            double lo = dt > 0 ? time[p] : t_end, hi = dt > 0 ? t_end : time[p];
            if (lo < fs->times[0] || hi > fs->times[fs->nt - 1]) return -1;
        }
    }
    if (nthreads < 1) nthreads = 1;
    if (nthreads > n) nthreads = (int)n;
    or_job *jobs = (or_job *)calloc((size_t)nthreads, sizeof(or_job));
    pthread_t *th = (pthread_t *)calloc((size_t)nthreads, sizeof(pthread_t));
    int64_t chunk = (n + nthreads - 1) / nthreads;
    for (int w = 0; w < nthreads; ++w) {
        or_job *jb = &jobs[w];
        jb->fs = fs; jb->kn = kn;
        jb->lon = lon; jb->lat = lat; jb->depth = depth; jb->time = time;
        jb->id = id; jb->step = step; jb->status = status;
        jb->age = age; jb->vars = vars; jb->hstep = hstep; jb->n = n;
        jb->dt = dt; jb->t_stop = t_stop; jb->t_end = t_end;
        jb->begin = (int64_t)w * chunk;
        jb->end = jb->begin + chunk < n ? jb->begin + chunk : n;
        if (jb->begin > n) jb->begin = n;
    }
    for (int w = 1; w < nthreads; ++w) pthread_create(&th[w], NULL, run_range, &jobs[w]);
    run_range(&jobs[0]);
    int64_t total = jobs[0].steps_done;
    for (int w = 1; w < nthreads; ++w) {
        pthread_join(th[w], NULL);
        total += jobs[w].steps_done;
    }
    free(jobs);
    free(th);
    return total;
}

/* ------------------------------------------------------------------------ */
/* Reduced-precision field storage (precision form): per (field, snapshot)   */
/* scale s = max|v| / (largest finite half / 2); stored q = round(v / s) to  */
/* binary16 or bfloat16 with round-to-nearest-even; value = q * s.           */
/* ------------------------------------------------------------------------ */

/* IEEE binary32 -> binary16, round to nearest even, from the bit layouts. */
uint16_t or_f32_to_f16(float x)
{
    uint32_t b;
    memcpy(&b, &x, 4);
    uint32_t sign = (b >> 16) & 0x8000u;
    int32_t exp = (int32_t)((b >> 23) & 0xFFu);
    uint32_t man = b & 0x7FFFFFu;
    if (exp == 0xFF) return (uint16_t)(sign | 0x7C00u | (man ? 0x200u : 0u));
    int32_t e = exp - 127 + 15;              /* biased binary16 exponent */
    if (e >= 0x1F) return (uint16_t)(sign | 0x7C00u);
    if (e <= 0) {                            /* subnormal or zero in binary16 */
        if (e < -10) return (uint16_t)sign;
        uint32_t m = man | 0x800000u;        /* 24-bit significand */
        int shift = 14 - e;                  /* 13 + (1 - e) */
        uint32_t q = m >> shift;
        uint32_t rem = m & ((1u << shift) - 1u);
        uint32_t halfway = 1u << (shift - 1);
        if (rem > halfway || (rem == halfway && (q & 1u))) q += 1u;
        return (uint16_t)(sign | q);
    }
    uint32_t q = ((uint32_t)e << 10) | (man >> 13);
    uint32_t rem = man & 0x1FFFu;
    if (rem > 0x1000u || (rem == 0x1000u && (q & 1u))) q += 1u;   /* may carry into exp */
    return (uint16_t)(sign | q);
}

double or_f16_to_f64(uint16_t h)
{
    int sign = (h >> 15) & 1;
    int exp = (h >> 10) & 0x1F;
    int man = h & 0x3FF;
    double v;
    if (exp == 0) v = ldexp((double)man, -24);
    else if (exp == 0x1F) v = man ? NAN : INFINITY;
    else v = ldexp((double)(man | 0x400), exp - 25);
    return sign ? -v : v;
}

/* IEEE binary32 -> bfloat16 (upper half of binary32), round to nearest even. */
uint16_t or_f32_to_bf16(float x)
{
    uint32_t b;
    memcpy(&b, &x, 4);
    if ((b & 0x7F800000u) == 0x7F800000u && (b & 0x7FFFFFu)) return (uint16_t)((b >> 16) | 0x40u);
    uint32_t lower = b & 0xFFFFu;
    uint32_t q = b >> 16;
    if (lower > 0x8000u || (lower == 0x8000u && (q & 1u))) q += 1u;
    return (uint16_t)q;
}

double or_bf16_to_f64(uint16_t h)
{
    uint32_t b = (uint32_t)h << 16;
    float f;
    memcpy(&f, &b, 4);
    return (double)f;
}

/* Quantise n values of one (field, snapshot) plane.  kind 0: binary16,
 * kind 1: bfloat16.  Returns the FP32 scale; q[i] = round(v[i] / s).  The
 * division is carried out in FP32, as the stored format is FP32-based. */
float or_quantise(const float *v, int64_t n, int kind, uint16_t *q)
{
    float amax = 0.0f;
    for (int64_t i = 0; i < n; ++i) {
        float a = fabsf(v[i]);
        if (a > amax) amax = a;
    }
    float s = amax > 0.0f ? amax / 32752.0f : 1.0f;
    for (int64_t i = 0; i < n; ++i) {
        float r = v[i] / s;
        q[i] = kind == 0 ? or_f32_to_f16(r) : or_f32_to_bf16(r);
    }
    return s;
}

/* Dequantise: value = q * s evaluated in FP32 (the stored representation),
 * then widened to FP64 for the oracle's arithmetic. */
void or_dequantise(const uint16_t *q, int64_t n, int kind, float s, double *out)
{
    for (int64_t i = 0; i < n; ++i) {
        float h = kind == 0 ? (float)or_f16_to_f64(q[i]) : (float)or_bf16_to_f64(q[i]);
        out[i] = (double)(h * s);
    }
}
