// sort.cu -- Morton re-sort with compaction, and FP64 moments.
//
// Re-sort: particles are bucketed by the Morton code of their (coarsened)
// cell indices, so that neighbouring threads advect particles in
// neighbouring cells and their field gathers share cache lines; deleted
// particles go to one last bucket behind all alive ones, so later launches
// cover only the alive prefix.  It is a counting sort: histogram, exclusive
// scan, scatter, then one gather of every particle array into the second set
// of arrays.  Order inside a bucket is not fixed; no particle's arithmetic
// depends on it.
//
// Moments: FP64 sums over alive particles, per block in a fixed order and
// then over blocks in a fixed order, so the result does not depend on timing.
#include "pg_host.h"

namespace pg {

namespace {

constexpr int kMaxKeyBits = 22;
constexpr int kScanBlock = 1024;
constexpr int kScanItems = 4;
constexpr int kScanTile = kScanBlock * kScanItems;

struct MortonSpec {
  int dims;
  int bits[3];
  int shift[3];
  int total;
};

// Bits of the Morton key: all cell bits of each axis, then the finest bits
// dropped (largest axis first) until the key has at most about twice as many
// buckets as particles (between 2^8 and 2^22 buckets).
MortonSpec morton_spec(const pg_fieldset *fs, int64_t n) {
  int max_bits = 1;
  while (max_bits < kMaxKeyBits && ((int64_t)1 << max_bits) < 2 * n) ++max_bits;
  if (max_bits < 8) max_bits = 8;
  MortonSpec m{};
  const int nodes[3] = {fs->nx, fs->ny, fs->nz};
  m.dims = fs->nz > 1 ? 3 : 2;
  m.total = 0;
  for (int d = 0; d < m.dims; ++d) {
    int b = 0;
    while ((1 << b) < nodes[d]) ++b;
    m.bits[d] = b;
    m.shift[d] = 0;
    m.total += b;
  }
  while (m.total > max_bits) {
    int w = 0;
    for (int d = 1; d < m.dims; ++d)
      if (m.bits[d] > m.bits[w]) w = d;
    --m.bits[w];
    ++m.shift[w];
    --m.total;
  }
  return m;
}

__device__ __forceinline__ int cell_index(const double *x, int n, int uni, double x0, double inv,
                                          double p) {
  int i;
  if (uni) {
    const double f = floor((p - x0) * inv);
    i = f < 0.0 ? 0 : (f > (double)(n - 1) ? n - 1 : (int)f);
  } else {
    int lo = 0, hi = n - 1;
    if (!(p >= x[0])) return 0;
    if (!(p < x[n - 1])) return n - 1;
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (x[mid] <= p) lo = mid; else hi = mid;
    }
    i = lo;
  }
  return i;
}

__device__ __forceinline__ uint32_t morton(const int (&c)[3], const MortonSpec &m) {
  uint32_t key = 0;
  int pos = 0;
  int maxb = 0;
  for (int d = 0; d < m.dims; ++d) maxb = m.bits[d] > maxb ? m.bits[d] : maxb;
  for (int b = 0; b < maxb; ++b)
    for (int d = 0; d < m.dims; ++d)
      if (b < m.bits[d]) key |= (uint32_t)(((c[d] >> m.shift[d]) >> b) & 1) << pos++;
  return key;
}

template <typename Real>
__global__ void bucket_kernel(GridArgs g, MortonSpec m, const Real *x, const Real *y,
                              const Real *z, const int32_t *ci, const int32_t *cj,
                              const int32_t *ck, const uint8_t *status, int64_t n,
                              uint32_t dead, uint32_t *key, uint32_t *count) {
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n;
       p += (int64_t)gridDim.x * blockDim.x) {
    uint32_t k = dead;
    if (status[p] == 0) {
      int c[3] = {0, 0, 0};
      if (ci) {
        c[0] = ci[p]; c[1] = cj[p]; c[2] = ck ? ck[p] : 0;
      } else {
        double lon = (double)x[p];
        if (g.periodic) {
          double r = fmod(lon - g.lon[0], 360.0);
          if (r < 0.0) r += 360.0;
          lon = g.lon[0] + r;
        }
        c[0] = cell_index(g.lon, g.nx, g.uni[0], g.x0[0], g.inv_d[0], lon);
        c[1] = cell_index(g.lat, g.ny, g.uni[1], g.x0[1], g.inv_d[1], (double)y[p]);
        if (g.nz > 1) c[2] = cell_index(g.depth, g.nz, g.uni[2], g.x0[2], g.inv_d[2], (double)z[p]);
      }
      k = morton(c, m);
    }
    key[p] = k;
    atomicAdd(&count[k], 1u);
  }
}

// Exclusive scan of m counts, tile by tile (1024 threads x 4 items).
__global__ void scan_tiles_kernel(const uint32_t *in, uint32_t *out, uint32_t *tile_sums,
                                  int64_t m) {
  __shared__ uint32_t s[kScanBlock];
  const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
  uint32_t v[kScanItems];
  uint32_t local = 0;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    v[i] = base + i < m ? in[base + i] : 0u;
    local += v[i];
  }
  s[threadIdx.x] = local;
  __syncthreads();
  for (int o = 1; o < kScanBlock; o <<= 1) {
    const uint32_t add = threadIdx.x >= (unsigned)o ? s[threadIdx.x - o] : 0u;
    __syncthreads();
    s[threadIdx.x] += add;
    __syncthreads();
  }
  uint32_t run = s[threadIdx.x] - local;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    if (base + i < m) out[base + i] = run;
    run += v[i];
  }
  if (threadIdx.x == kScanBlock - 1) tile_sums[blockIdx.x] = s[threadIdx.x];
}

__global__ void scan_add_kernel(uint32_t *out, const uint32_t *tile_off, int64_t m) {
  const int64_t base = (int64_t)blockIdx.x * kScanTile;
  const uint32_t add = tile_off[blockIdx.x];
  for (int i = threadIdx.x; i < kScanTile; i += blockDim.x)
    if (base + i < m) out[base + i] += add;
}

__global__ void scatter_kernel(const uint32_t *key, uint32_t *offset, uint32_t *perm, int64_t n) {
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n;
       p += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t at = atomicAdd(&offset[key[p]], 1u);
    perm[at] = (uint32_t)p;
  }
}

template <typename T>
__global__ void gather_kernel(const T *src, T *dst, const uint32_t *perm, int64_t n) {
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n;
       p += (int64_t)gridDim.x * blockDim.x)
    dst[p] = src[perm[p]];
}

int grid_of(int64_t n, int sm) {
  int64_t g = (n + 255) / 256;
  if (g > (int64_t)sm * 32) g = (int64_t)sm * 32;
  return (int)(g < 1 ? 1 : g);
}

// Exclusive scan of m entries in place of `out` (in may equal out).
cudaError_t exclusive_scan(const uint32_t *in, uint32_t *out, int64_t m, uint32_t *tmp,
                           cudaStream_t st) {
  const int64_t tiles = (m + kScanTile - 1) / kScanTile;
  uint32_t *sums = tmp;                 // [tiles]
  uint32_t *sums_out = tmp + tiles;     // [tiles]
  uint32_t *dummy = tmp + 2 * tiles;    // [1]
  scan_tiles_kernel<<<(unsigned)tiles, kScanBlock, 0, st>>>(in, out, sums, m);
  if (tiles > 1) {
    // tiles <= kScanTile, so one tile scans all tile sums
    scan_tiles_kernel<<<1, kScanBlock, 0, st>>>(sums, sums_out, dummy, tiles);
    scan_add_kernel<<<(unsigned)tiles, 256, 0, st>>>(out, sums_out, m);
    note_launches(2);
  }
  note_launches(1);
  return cudaGetLastError();
}

}  // namespace

// Exclusive scan of m 32-bit entries (m at most scan_max_entries()) with a
// scratch of scan_scratch_words(m) words; in may equal out.
int64_t scan_max_entries() { return (int64_t)kScanTile * kScanTile; }
size_t scan_scratch_words(int64_t m) { return (size_t)(2 * ((m + kScanTile - 1) / kScanTile) + 1); }
cudaError_t exclusive_scan_u32(const uint32_t *in, uint32_t *out, int64_t m, uint32_t *tmp,
                               cudaStream_t st) {
  if (m <= 0) return cudaSuccess;
  if (m > scan_max_entries()) return cudaErrorInvalidValue;
  return exclusive_scan(in, out, m, tmp, st);
}

// n_alive == nullptr: keep the particle arrays where they are (the sorted
// copy is copied back) and read nothing back to the host, so the whole
// re-sort is a fixed sequence of device operations (capturable in a graph).
// Scratch and the second array set must then already exist
// (prepare_resort).
cudaError_t prepare_resort(pg_pset *ps) {
  const int64_t n = ps->n;
  if (n == 0) return cudaSuccess;
  const MortonSpec m = morton_spec(ps->fs, n);
  const int64_t nb = ((int64_t)1 << m.total) + 1;
  const int64_t tiles = (nb + kScanTile - 1) / kScanTile;
  const size_t need = sizeof(uint32_t) * ((size_t)n * 2 + (size_t)nb * 2 + (size_t)tiles * 2 + 1);
  cudaError_t e;
  if (ps->sort_scratch_bytes < need) {
    dev_free(ps->sort_scratch);
    ps->sort_scratch = nullptr;
    ps->sort_scratch_bytes = 0;
    if ((e = dev_alloc(&ps->sort_scratch, need)) != cudaSuccess) return e;
    ps->sort_scratch_bytes = need;
  }
  // the second set has exactly the first one's capacity: the sampled
  // variables are laid out with the capacity as their stride
  if (ps->alt_cap != ps->cap) {
    ps->alt.free_all();
    ps->alt_cap = 0;
    if (alloc_arrays(ps->alt, ps->pos, ps->cap, ps->nvar) != PG_OK)
      return cudaErrorMemoryAllocation;
    ps->alt_cap = ps->cap;
  }
  return cudaSuccess;
}

cudaError_t launch_resort(pg_pset *ps, cudaStream_t st, int64_t *n_alive) {
  const int64_t n = ps->n;
  if (n_alive) *n_alive = n;
  if (n == 0) return cudaSuccess;
  if (n >= (int64_t)0xFFFFFFFFll) return cudaErrorInvalidValue;
  const pg_fieldset *fs = ps->fs;
  const MortonSpec m = morton_spec(fs, n);
  const uint32_t dead = 1u << m.total;
  const int64_t nb = (int64_t)dead + 1;
  cudaError_t e;
  if ((e = prepare_resort(ps)) != cudaSuccess) return e;
  uint32_t *key = (uint32_t *)ps->sort_scratch;
  uint32_t *perm = key + n;
  uint32_t *count = perm + n;
  uint32_t *offset = count + nb;
  uint32_t *tmp = offset + nb;
  const int sm = fs->sm_count;
  GridArgs g;
  g.nx = fs->nx; g.ny = fs->ny; g.nz = fs->nz; g.mesh = fs->mesh; g.periodic = fs->periodic;
  g.lon = fs->d_axes64; g.lat = fs->d_axes64 + fs->nx; g.depth = fs->d_axes64 + fs->nx + fs->ny;
  for (int a = 0; a < 3; ++a) { g.uni[a] = fs->uni[a]; g.x0[a] = fs->x0[a]; g.inv_d[a] = fs->inv_d[a]; }
  if ((e = cudaMemsetAsync(count, 0, sizeof(uint32_t) * nb, st)) != cudaSuccess) return e;
  const int gr = grid_of(n, sm);
  if (ps->pos == PG_POS_F64)
    bucket_kernel<double><<<gr, 256, 0, st>>>(g, m, (const double *)ps->x, (const double *)ps->y,
                                              (const double *)ps->z, nullptr, nullptr, nullptr,
                                              ps->status, n, dead, key, count);
  else if (ps->pos == PG_POS_F32)
    bucket_kernel<float><<<gr, 256, 0, st>>>(g, m, (const float *)ps->x, (const float *)ps->y,
                                             (const float *)ps->z, nullptr, nullptr, nullptr,
                                             ps->status, n, dead, key, count);
  else
    bucket_kernel<float><<<gr, 256, 0, st>>>(g, m, nullptr, nullptr, nullptr, ps->ci, ps->cj,
                                             fs->nz > 1 ? ps->ck : nullptr, ps->status, n, dead,
                                             key, count);
  note_launches(1);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if ((e = exclusive_scan(count, offset, nb, tmp, st)) != cudaSuccess) return e;
  uint32_t dead_count = 0;
  if (n_alive &&
      (e = cudaMemcpyAsync(&dead_count, count + dead, 4, cudaMemcpyDeviceToHost, st)) != cudaSuccess)
    return e;
  scatter_kernel<<<gr, 256, 0, st>>>(key, offset, perm, n);
  PsetArrays &B = ps->alt;
  if (ps->pos == PG_POS_CELL) {
    gather_kernel<int32_t><<<gr, 256, 0, st>>>(ps->ci, B.ci, perm, n);
    gather_kernel<int32_t><<<gr, 256, 0, st>>>(ps->cj, B.cj, perm, n);
    gather_kernel<int32_t><<<gr, 256, 0, st>>>(ps->ck, B.ck, perm, n);
    gather_kernel<float><<<gr, 256, 0, st>>>(ps->fx, B.fx, perm, n);
    gather_kernel<float><<<gr, 256, 0, st>>>(ps->fy, B.fy, perm, n);
    gather_kernel<float><<<gr, 256, 0, st>>>(ps->fz, B.fz, perm, n);
  } else if (ps->pos == PG_POS_F64) {
    gather_kernel<double><<<gr, 256, 0, st>>>((const double *)ps->x, (double *)B.x, perm, n);
    gather_kernel<double><<<gr, 256, 0, st>>>((const double *)ps->y, (double *)B.y, perm, n);
    gather_kernel<double><<<gr, 256, 0, st>>>((const double *)ps->z, (double *)B.z, perm, n);
  } else {
    gather_kernel<float><<<gr, 256, 0, st>>>((const float *)ps->x, (float *)B.x, perm, n);
    gather_kernel<float><<<gr, 256, 0, st>>>((const float *)ps->y, (float *)B.y, perm, n);
    gather_kernel<float><<<gr, 256, 0, st>>>((const float *)ps->z, (float *)B.z, perm, n);
  }
  gather_kernel<double><<<gr, 256, 0, st>>>(ps->time, B.time, perm, n);
  gather_kernel<uint64_t><<<gr, 256, 0, st>>>(ps->id, B.id, perm, n);
  gather_kernel<uint32_t><<<gr, 256, 0, st>>>(ps->step, B.step, perm, n);
  gather_kernel<uint8_t><<<gr, 256, 0, st>>>(ps->status, B.status, perm, n);
  gather_kernel<double><<<gr, 256, 0, st>>>(ps->age, B.age, perm, n);
  gather_kernel<double><<<gr, 256, 0, st>>>(ps->hstep, B.hstep, perm, n);
  for (int j = 0; j < ps->nvar; ++j)
    gather_kernel<double><<<gr, 256, 0, st>>>(ps->var + (size_t)j * ps->cap,
                                              B.var + (size_t)j * ps->cap, perm, n);
  note_launches((ps->pos == PG_POS_CELL ? 11 : 8) + 2 + ps->nvar);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if (!n_alive) {
    // fixed-pointer mode: copy the sorted arrays back in place
    const auto arrays_a = std::vector<std::pair<void *, void *>>{
        {ps->x, B.x}, {ps->y, B.y}, {ps->z, B.z}, {ps->ci, B.ci}, {ps->cj, B.cj},
        {ps->ck, B.ck}, {ps->fx, B.fx}, {ps->fy, B.fy}, {ps->fz, B.fz}};
    const size_t el = ps->pos == PG_POS_F64 ? 8 : 4;
    for (const auto &pr : arrays_a)
      if (pr.first && (e = cudaMemcpyAsync(pr.first, pr.second, (size_t)n * el,
                                           cudaMemcpyDeviceToDevice, st)) != cudaSuccess)
        return e;
    if ((e = cudaMemcpyAsync(ps->time, B.time, (size_t)n * 8, cudaMemcpyDeviceToDevice, st)) ||
        (e = cudaMemcpyAsync(ps->id, B.id, (size_t)n * 8, cudaMemcpyDeviceToDevice, st)) ||
        (e = cudaMemcpyAsync(ps->step, B.step, (size_t)n * 4, cudaMemcpyDeviceToDevice, st)) ||
        (e = cudaMemcpyAsync(ps->status, B.status, (size_t)n, cudaMemcpyDeviceToDevice, st)) ||
        (e = cudaMemcpyAsync(ps->age, B.age, (size_t)n * 8, cudaMemcpyDeviceToDevice, st)) ||
        (e = cudaMemcpyAsync(ps->hstep, B.hstep, (size_t)n * 8, cudaMemcpyDeviceToDevice, st)))
      return e;
    for (int j = 0; j < ps->nvar; ++j)
      if ((e = cudaMemcpyAsync(ps->var + (size_t)j * ps->cap, B.var + (size_t)j * ps->cap,
                               (size_t)n * 8, cudaMemcpyDeviceToDevice, st)) != cudaSuccess)
        return e;
    return cudaSuccess;
  }
  // swap the two array sets
  const PsetArrays A = pset_arrays(ps);
  pset_set_arrays(ps, B);
  B = A;
  if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return e;
  *n_alive = n - (int64_t)dead_count;
  return cudaSuccess;
}

// ----------------------------------------------------------------- moments

namespace {

constexpr int kMomBlocks = 256;
constexpr int kMomThreads = 256;

template <typename Real>
__device__ __forceinline__ void pos_of(const Real *x, const Real *y, const Real *z,
                                       const int32_t *ci, const int32_t *cj, const int32_t *ck,
                                       const float *fx, const float *fy, const float *fz,
                                       const GridArgs &g, int64_t p, double &a, double &b,
                                       double &c) {
  if (ci) {   // uniform axes: x0 + (index + offset) * spacing
    a = g.x0[0] + ((double)ci[p] + (double)fx[p]) * g.d[0];
    b = g.x0[1] + ((double)cj[p] + (double)fy[p]) * g.d[1];
    c = ck ? g.x0[2] + ((double)ck[p] + (double)fz[p]) * g.d[2] : 0.0;
  } else {
    a = (double)x[p]; b = (double)y[p]; c = (double)z[p];
  }
}

// Block b sums the contiguous range [b*chunk, (b+1)*chunk) in index order,
// thread-strided, then combines threads in a fixed tree.
template <typename Real>
__global__ void moments_kernel(GridArgs g, const Real *x, const Real *y, const Real *z,
                               const int32_t *ci, const int32_t *cj, const int32_t *ck,
                               const float *fx, const float *fy, const float *fz,
                               const uint8_t *status, int64_t n, double *partial) {
  __shared__ double sh[7][kMomThreads];
  const int64_t chunk = (n + gridDim.x - 1) / gridDim.x;
  const int64_t beg = (int64_t)blockIdx.x * chunk;
  const int64_t end = beg + chunk < n ? beg + chunk : n;
  double acc[7] = {0, 0, 0, 0, 0, 0, 0};
  for (int64_t p = beg + threadIdx.x; p < end; p += blockDim.x) {
    if (status[p] != 0) continue;
    double a, b, c;
    pos_of<Real>(x, y, z, ci, cj, ck, fx, fy, fz, g, p, a, b, c);
    acc[0] += 1.0; acc[1] += a; acc[2] += b; acc[3] += c;
    acc[4] += a * a; acc[5] += b * b; acc[6] += c * c;
  }
  for (int q = 0; q < 7; ++q) sh[q][threadIdx.x] = acc[q];
  __syncthreads();
  for (int o = kMomThreads / 2; o > 0; o >>= 1) {
    if (threadIdx.x < (unsigned)o)
      for (int q = 0; q < 7; ++q) sh[q][threadIdx.x] += sh[q][threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0)
    for (int q = 0; q < 7; ++q) partial[blockIdx.x * 7 + q] = sh[q][0];
}

__global__ void moments_final_kernel(const double *partial, int nblocks, double *out) {
  const int q = threadIdx.x;
  if (q < 7) {
    double s = 0.0;
    for (int b = 0; b < nblocks; ++b) s += partial[b * 7 + q];
    out[q] = s;
  }
}

}  // namespace

cudaError_t launch_moments(const pg_pset *ps_c, double *out7, cudaStream_t st) {
  pg_pset *ps = const_cast<pg_pset *>(ps_c);
  cudaError_t e;
  if (!ps->diag_scratch) {
    if ((e = dev_alloc((void **)&ps->diag_scratch, sizeof(double) * (kMomBlocks * 7 + 8))) !=
        cudaSuccess)
      return e;
  }
  const pg_fieldset *fs = ps->fs;
  const GridArgs g = grid_args_of(fs);
  double *partial = ps->diag_scratch;
  double *res = partial + kMomBlocks * 7;
  const int64_t n = ps->n;
  if (ps->pos == PG_POS_F64)
    moments_kernel<double><<<kMomBlocks, kMomThreads, 0, st>>>(
        g, (const double *)ps->x, (const double *)ps->y, (const double *)ps->z, nullptr, nullptr,
        nullptr, nullptr, nullptr, nullptr, ps->status, n, partial);
  else if (ps->pos == PG_POS_F32)
    moments_kernel<float><<<kMomBlocks, kMomThreads, 0, st>>>(
        g, (const float *)ps->x, (const float *)ps->y, (const float *)ps->z, nullptr, nullptr,
        nullptr, nullptr, nullptr, nullptr, ps->status, n, partial);
  else
    moments_kernel<float><<<kMomBlocks, kMomThreads, 0, st>>>(
        g, nullptr, nullptr, nullptr, ps->ci, ps->cj, fs->nz > 1 ? ps->ck : nullptr, ps->fx,
        ps->fy, fs->nz > 1 ? ps->fz : nullptr, ps->status, n, partial);
  moments_final_kernel<<<1, 32, 0, st>>>(partial, kMomBlocks, res);
  note_launches(2);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if ((e = cudaMemcpyAsync(out7, res, sizeof(double) * 7, cudaMemcpyDeviceToHost, st)) != cudaSuccess)
    return e;
  return cudaStreamSynchronize(st);
}

}  // namespace pg
