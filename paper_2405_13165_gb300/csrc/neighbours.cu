// neighbours.cu -- fixed-radius neighbour search of Eq. Nbd (Sec. 2.2) on a
// cell list: bounding box -> cell keys -> stable LSD radix sort -> cell ranges
// -> count (one block per occupied cell, candidate tiles staged in shared
// memory) -> exclusive scan -> fill -> (row sort when the input order is not
// the cell order) ; plus the transpose map used by the apply adjoint.
#include <algorithm>
#include <climits>

#include "internal.cuh"

namespace mafp {

// ---------------------------------------------------------------- grid set-up
constexpr int kBoxThreads = 256;
constexpr int kBoxBlocks = 16384;   // bounding-box blocks over all clouds
constexpr int kBoxPartsMax = 1024;  // blocks of one cloud

// ------------------------------------------------ several clouds, one grid each
// Cloud b owns particles [off[b], off[b+1]) and cells [cell_base[b], cell_base[b+1])
// of the global cell numbering, with its own bounding box and cell edge, so
// neighbourhoods never cross clouds.  A single cloud is the case nb = 1.
struct CloudGrids {
  const GridDev *grids;      // [nb]
  const long long *cell_base;  // [nb + 1]
  int nb;
  const GridDev *all;        // ok flag and total cell count
};

__global__ void k_set_one_cloud(long long *off, int64_t n) {
  off[0] = 0;
  off[1] = n;
}

// Block (b, part) reduces part `part` of cloud b: min / max of x, y, z, max h,
// count of non-finite entries; also records each particle's cloud.  Min and
// max are exact in the input's own type, so they are taken in it and widened
// once per block.
template <typename T>
__device__ __forceinline__ T lo_of(T a, T b) { return b < a ? b : a; }
template <typename T>
__device__ __forceinline__ T hi_of(T a, T b) { return b > a ? b : a; }

template <typename T>
__global__ void __launch_bounds__(kBoxThreads) k_cloud_bbox(const vec4_t<T> *pos, int64_t n,
                                                            const long long *off, int nb,
                                                            int parts, double *partial,
                                                            int32_t *cloud_id) {
  const int b = blockIdx.x / parts, part = blockIdx.x % parts;
  // offsets are checked in k_cloud_grid; clamping keeps every access in [0, n)
  const long long lo = max(0LL, min(off[b], (long long)n));
  const long long hi = max(lo, min(off[b + 1], (long long)n));
  const T inf = T(INFINITY);
  T v[7] = {inf, inf, inf, -inf, -inf, -inf, T(0)};
  int bad = 0;
  for (long long i = lo + (long long)part * blockDim.x + threadIdx.x; i < hi;
       i += (long long)parts * blockDim.x) {
    cloud_id[i] = b;
    const vec4_t<T> p = ld4(pos + i);
    const bool ok = isfinite(p.x) && isfinite(p.y) && isfinite(p.z) && isfinite(p.w) && p.w > T(0);
    if (!ok) {
      ++bad;
      continue;
    }
    v[0] = lo_of(v[0], p.x); v[1] = lo_of(v[1], p.y); v[2] = lo_of(v[2], p.z);
    v[3] = hi_of(v[3], p.x); v[4] = hi_of(v[4], p.y); v[5] = hi_of(v[5], p.z);
    v[6] = hi_of(v[6], p.w);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
    for (int k = 0; k < 3; ++k) v[k] = lo_of(v[k], __shfl_xor_sync(0xffffffffu, v[k], o));
#pragma unroll
    for (int k = 3; k < 7; ++k) v[k] = hi_of(v[k], __shfl_xor_sync(0xffffffffu, v[k], o));
    bad += __shfl_xor_sync(0xffffffffu, bad, o);
  }
  __shared__ T red[kBoxThreads / 32][7];
  __shared__ int red_bad[kBoxThreads / 32];
  if ((threadIdx.x & 31) == 0) {
    for (int k = 0; k < 7; ++k) red[threadIdx.x >> 5][k] = v[k];
    red_bad[threadIdx.x >> 5] = bad;
  }
  __syncthreads();
  if (threadIdx.x < 8) {
    const int k = threadIdx.x;
    double a;
    if (k < 7) {
      T r = red[0][k];
      for (int w = 1; w < kBoxThreads / 32; ++w)
        r = k < 3 ? lo_of(r, red[w][k]) : hi_of(r, red[w][k]);
      a = (double)r;
    } else {
      int s = 0;
      for (int w = 0; w < kBoxThreads / 32; ++w) s += red_bad[w];
      a = (double)s;
    }
    partial[(long long)blockIdx.x * 8 + k] = a;
  }
}

// One warp per cloud folds the cloud's `parts` partials (lanes over parts,
// then shuffles) and leaves the cloud's box in its first partial slot.
__global__ void __launch_bounds__(kBoxThreads) k_cloud_fold(double *partial, int nb, int parts) {
  const int lane = threadIdx.x & 31;
  const int b = blockIdx.x * (kBoxThreads / 32) + (threadIdx.x >> 5);
  if (b >= nb) return;
  double v[8] = {INFINITY, INFINITY, INFINITY, -INFINITY, -INFINITY, -INFINITY, 0.0, 0.0};
  double *pb = partial + (long long)b * parts * 8;
  for (int q = lane; q < parts; q += 32)
    for (int k = 0; k < 8; ++k) {
      const double a = pb[q * 8 + k];
      v[k] = k < 3 ? fmin(v[k], a) : (k < 7 ? fmax(v[k], a) : v[k] + a);
    }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
    for (int k = 0; k < 3; ++k) v[k] = fmin(v[k], __shfl_xor_sync(0xffffffffu, v[k], o));
#pragma unroll
    for (int k = 3; k < 7; ++k) v[k] = fmax(v[k], __shfl_xor_sync(0xffffffffu, v[k], o));
    v[7] += __shfl_xor_sync(0xffffffffu, v[7], o);
  }
  __syncwarp();
  if (lane == 0)
    for (int k = 0; k < 8; ++k) pb[k] = v[k];
}

// Cells of cloud b at edge c (>= max h of the cloud); 0 for an empty cloud.
__device__ double cloud_cells(const double v[8], double c, int dim[3]) {
  if (!(v[6] > 0.0)) {
    dim[0] = dim[1] = dim[2] = 1;
    return 0.0;
  }
  double cells = 1.0;
  for (int a = 0; a < 3; ++a) {
    const double d = floor((v[3 + a] - v[a]) / c) + 1.0;
    cells *= d;
    dim[a] = d < 2e9 ? (int)d : INT_MAX;
  }
  return cells;
}

// One block: per-cloud grids from the folded boxes, the global cell numbering
// (exclusive scan of the clouds' cell counts) and the all-clouds flag.  The cell
// edge of every cloud starts strictly above its max h times edge_factor >= 1
// (so S_i lies in the 27 cells around i's cell) and grows uniformly when the
// total exceeds cap_cells.
__global__ void __launch_bounds__(kBoxThreads) k_cloud_grid(double *partial,
                                                            const long long *off, int64_t n,
                                                            int nb, int parts, GridDev *grids,
                                                            long long *cell_base, GridDev *all,
                                                            DevStatus *st, long long cap_cells,
                                                            double edge_factor) {
  __shared__ double s_nonfinite, s_cells;
  __shared__ double s_scale;
  __shared__ int s_bad;
  __shared__ long long s_sum[kBoxThreads];
  if (threadIdx.x == 0) {
    s_nonfinite = 0.0;
    s_scale = 1.0;
    s_bad = (off[0] != 0 || off[nb] != n) ? 1 : 0;
  }
  __syncthreads();
  for (int b = threadIdx.x; b < nb; b += blockDim.x)
    if (off[b + 1] < off[b]) s_bad = 1;
  __syncthreads();
  if (s_bad) {
    // the offsets do not split [0, n) into consecutive ranges
    if (threadIdx.x == 0) {
      all->ok = 0;
      set_error(st, MAFP_EINVAL, -1);
    }
    return;
  }
  for (int b = threadIdx.x; b < nb; b += blockDim.x) {
    const double bad = partial[(long long)b * parts * 8 + 7];
    if (bad > 0.0) atomicAdd(&s_nonfinite, bad);
  }
  __syncthreads();
  if (s_nonfinite > 0.0) {
    if (threadIdx.x == 0) {
      all->ok = 0;
      st->n_nonfinite += (long long)s_nonfinite;
      set_error(st, MAFP_ENONFINITE, (long long)s_nonfinite);
    }
    return;
  }
  for (int it = 0; it < 64; ++it) {
    if (threadIdx.x == 0) s_cells = 0.0;
    __syncthreads();
    for (int b = threadIdx.x; b < nb; b += blockDim.x) {
      double v[8];
      for (int k = 0; k < 8; ++k) v[k] = partial[(long long)b * parts * 8 + k];
      int dim[3];
      const double c = v[6] * (1.0 + 1e-6) * edge_factor * s_scale;
      const double cells = cloud_cells(v, c, dim);
      GridDev &g = grids[b];
      for (int a = 0; a < 3; ++a) g.lo[a] = v[a] < INFINITY ? v[a] : 0.0;
      g.hmax = v[6];
      g.c = c;
      g.inv_c = v[6] > 0.0 ? 1.0 / c : 1.0;
      for (int a = 0; a < 3; ++a) g.dim[a] = dim[a];
      g.ncells = (long long)cells;
      g.ok = 1;
      atomicAdd(&s_cells, cells);
    }
    __syncthreads();
    const bool fits = s_cells <= (double)cap_cells;
    __syncthreads();
    if (fits) break;
    if (threadIdx.x == 0) s_scale *= cbrt(s_cells / (double)cap_cells) * 1.0001;
    __syncthreads();
  }
  // exclusive scan of the cell counts: thread t takes a contiguous chunk
  const int chunk = (nb + kBoxThreads - 1) / kBoxThreads;
  const int b0 = threadIdx.x * chunk, b1 = min(nb, b0 + chunk);
  long long part_sum = 0;
  for (int b = b0; b < b1; ++b) part_sum += grids[b].ncells;
  s_sum[threadIdx.x] = part_sum;
  __syncthreads();
  if (threadIdx.x == 0) {
    long long acc = 0;
    for (int t = 0; t < kBoxThreads; ++t) {
      const long long v = s_sum[t];
      s_sum[t] = acc;
      acc += v;
    }
  }
  __syncthreads();
  long long run = s_sum[threadIdx.x];
  for (int b = b0; b < b1; ++b) {
    cell_base[b] = run;
    run += grids[b].ncells;
  }
  if (threadIdx.x == 0) {
    long long acc = s_sum[kBoxThreads - 1];
    for (int b = (kBoxThreads - 1) * chunk; b < nb; ++b) acc += grids[b].ncells;
    cell_base[nb] = acc;
    all->ok = acc <= cap_cells ? 1 : 0;
    all->ncells = acc;
    all->c = grids[0].c;
    if (acc > cap_cells) set_error(st, MAFP_ECAPACITY, cap_cells);
    st->ncells = acc;
    st->cell_size = grids[0].c;
    st->not_identity = 0;
  }
}

template <typename T>
__global__ void k_hash(const vec4_t<T> *pos, int64_t n, const int32_t *cloud_id, CloudGrids cg,
                       uint32_t *keys, int32_t *vals) {
  if (!cg.all->ok) return;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int b = cloud_id[i];
    const GridDev &g = cg.grids[b];
    vec4_t<T> p = ld4(pos + i);
    double q[3] = {(double)p.x, (double)p.y, (double)p.z};
    long long c[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      long long v = (long long)floor((q[a] - g.lo[a]) * g.inv_c);
      v = v < 0 ? 0 : (v >= g.dim[a] ? g.dim[a] - 1 : v);
      c[a] = v;
    }
    keys[i] = (uint32_t)(cg.cell_base[b] + (c[2] * g.dim[1] + c[1]) * g.dim[0] + c[0]);
    vals[i] = (int32_t)i;
  }
}

__global__ void k_clear_cells(const GridDev *g, int32_t *cell_start, int32_t *cell_end,
                              int32_t *n_ucell) {
  if (!g->ok) return;
  const long long nc = g->ncells;
  // occupied cells, overflow cells, and the work tickets of the mask and fill kernels
  if (blockIdx.x == 0 && threadIdx.x == 0)
    n_ucell[0] = n_ucell[1] = n_ucell[2] = n_ucell[3] = n_ucell[4] = 0;
  for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < nc;
       k += (long long)gridDim.x * blockDim.x) {
    cell_start[k] = INT_MAX;
    cell_end[k] = 0;
  }
}

// ------------------------------------------------------------- radix sort
constexpr int kRadixThreads = 256;
constexpr int kRadixItems = 8;
constexpr int kRadixTile = kRadixThreads * kRadixItems;

__global__ void __launch_bounds__(kRadixThreads) k_radix_hist(const uint32_t *keys, int64_t n,
                                                              int shift, int32_t *hist,
                                                              int tiles, const GridDev *g) {
  if (!g->ok) return;
  __shared__ int32_t cnt[256];
  cnt[threadIdx.x] = 0;
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * kRadixTile;
  for (int k = threadIdx.x; k < kRadixTile; k += kRadixThreads) {
    int64_t idx = base + k;
    if (idx < n) atomicAdd(&cnt[(keys[idx] >> shift) & 255u], 1);
  }
  __syncthreads();
  hist[(int64_t)threadIdx.x * tiles + blockIdx.x] = cnt[threadIdx.x];
}

__global__ void __launch_bounds__(kRadixThreads) k_radix_scatter(
    const uint32_t *kin, const int32_t *vin, uint32_t *kout, int32_t *vout, int64_t n, int shift,
    const long long *offs, int tiles, const GridDev *g) {
  if (!g->ok) return;
  __shared__ long long base_d[256];
  __shared__ int32_t wcnt[kRadixThreads / 32][256];
  __shared__ int32_t ctot[256];
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  base_d[tid] = offs[(int64_t)tid * tiles + blockIdx.x];
  const unsigned lt = (1u << lane) - 1u;
  for (int c = 0; c < kRadixItems; ++c) {
    for (int k = tid; k < (kRadixThreads / 32) * 256; k += kRadixThreads) (&wcnt[0][0])[k] = 0;
    __syncthreads();
    const int64_t idx = (int64_t)blockIdx.x * kRadixTile + (int64_t)c * kRadixThreads + tid;
    const bool valid = idx < n;
    uint32_t key = valid ? kin[idx] : 0u;
    int32_t val = valid ? vin[idx] : 0;
    int d = valid ? (int)((key >> shift) & 255u) : 256;
    unsigned peers = __match_any_sync(0xffffffffu, d);
    int rank = __popc(peers & lt);
    if (valid && rank == 0) wcnt[w][d] = __popc(peers);
    __syncthreads();
    {
      int run = 0;
      for (int ww = 0; ww < kRadixThreads / 32; ++ww) {
        int t = wcnt[ww][tid];
        wcnt[ww][tid] = run;
        run += t;
      }
      ctot[tid] = run;
    }
    __syncthreads();
    if (valid) {
      long long p = base_d[d] + wcnt[w][d] + rank;
      kout[p] = key;
      vout[p] = val;
    }
    __syncthreads();
    base_d[tid] += ctot[tid];
    __syncthreads();
  }
}

// Exclusive scan of the (digit-major) histogram; reuses the int32->int64 scan.
// --------------------------------------------------------- cell ranges
// Occupied cells go to the work queue in two groups, the ones holding at least
// kBigCell particles (3D cells at the usual h / dx) ahead of the rest, so the
// costly cells are taken first and the kernels end on cheap ones.
constexpr int kBigCell = 24;
// Slot of the cell with ticket t: the first n_ucell[0] tickets are the front
// group, the n_ucell[4] after them the back group (stored from slot n - 1 down).
__device__ __forceinline__ int cell_slot(int t, int nbig, int64_t n) {
  return t < nbig ? t : (int)(n - 1 - (t - nbig));
}
template <typename T>
__global__ void k_cells(const uint32_t *skeys, const int32_t *svals, int64_t n,
                        const vec4_t<T> *pos, vec4_t<T> *spos, int32_t *cell_start,
                        int32_t *cell_end, int32_t *ucell, int32_t *n_ucell, DevStatus *st,
                        int32_t *order, const GridDev *g) {
  if (!g->ok) return;
  for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < n;
       s += (int64_t)gridDim.x * blockDim.x) {
    uint32_t key = skeys[s];
    int32_t i = svals[s];
    st4(spos + s, ld4(pos + i));
    if (order) order[s] = i;
    if (i != (int32_t)s) st->not_identity = 1;
    if (s == 0 || skeys[s - 1] != key) {
      cell_start[key] = (int32_t)s;
      // the work queue of the mask and fill kernels, costly cells first: cells
      // of at least kBigCell particles fill the list from the front, the others
      // from the back (slot n - 1 - u; there are at most n cells)
      const bool big = s + kBigCell - 1 < n && skeys[s + kBigCell - 1] == key;
      const int64_t u = big ? (int64_t)atomicAdd(n_ucell, 1)
                            : n - 1 - (int64_t)atomicAdd(n_ucell + 4, 1);
      ucell[2 * u] = (int32_t)key;
      ucell[2 * u + 1] = (int32_t)s;
    }
    if (s == n - 1 || skeys[s + 1] != key) cell_end[key] = (int32_t)(s + 1);
  }
}

__global__ void k_identity_flag(DevStatus *st) {
  st->cells_identity = st->not_identity ? 0 : 1;
}

// --------------------------------------------------------- count / fill
__device__ __forceinline__ bool in_support64(double xi, double yi, double zi, double hi,
                                             double xj, double yj, double zj, double hj) {
  double dx = __dsub_rn(xj, xi), dy = __dsub_rn(yj, yi), dz = __dsub_rn(zj, zi);
  double d2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
  double r = __dmul_rn(__dadd_rn(hi, hj), 0.5);
  return d2 <= __dmul_rn(r, r);
}

// FP32 decision, retaken in FP64 within a 1e-5 relative band of the bound.
__device__ __forceinline__ bool in_support(const float4 &a, const float4 &b) {
  float dx = b.x - a.x, dy = b.y - a.y, dz = b.z - a.z;
  float d2 = (dx * dx + dy * dy) + dz * dz;
  float r = (a.w + b.w) * 0.5f;
  float r2 = r * r;
  float diff = d2 - r2;
  if (fabsf(diff) <= 1e-5f * r2)
    return in_support64(a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w);
  return diff < 0.0f;
}
__device__ __forceinline__ bool in_support(const double4_16a &a, const double4_16a &b) {
  return in_support64(a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w);
}

constexpr int kNbrThreads = 128;
constexpr int kNbrSmemBytes = 32768;

// Warp-per-particle count / fill (ballot compaction), for the occupied cells
// listed in sel[0 .. *n_sel): the cells whose 27-cell candidate union does not
// fit the shared-memory tile of the mask kernel below.
struct CloudGrids;
__device__ __forceinline__ void cell_runs(int key, const CloudGrids &cg,
                                          const int32_t *cell_start, const int32_t *cell_end,
                                          int r, int *lo_out, int *len_out);

template <typename T, bool FILL>
__global__ void __launch_bounds__(kNbrThreads) k_nbr(
    CloudGrids cg, const int32_t *ucell, const int32_t *sel, const int32_t *n_sel,
    const vec4_t<T> *spos, const int32_t *svals, const int32_t *cell_start,
    const int32_t *cell_end, int32_t *counts, const long long *row_ptr, int32_t *col,
    long long cap_nnz, int64_t n) {
  using V = vec4_t<T>;
  constexpr int CAP = kNbrSmemBytes / sizeof(V);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  V *cand = reinterpret_cast<V *>(smem_raw);
  __shared__ int r_lo[9], r_len[9], r_off[10];
  if (!cg.all->ok) return;
  if (FILL && row_ptr[n] > cap_nnz) return;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = kNbrThreads / 32;
  const unsigned lt = (1u << lane) - 1u;
  const int nu = *n_sel;
  for (int cs = blockIdx.x; cs < nu; cs += gridDim.x) {
    const int cb = sel[cs];
    const int key = ucell[2 * cb], s0 = ucell[2 * cb + 1];
    const int s1 = cell_end[key];
    if (threadIdx.x < 9)
      cell_runs(key, cg, cell_start, cell_end, threadIdx.x, &r_lo[threadIdx.x], &r_len[threadIdx.x]);
    __syncthreads();
    if (threadIdx.x == 0) {
      int o = 0;
      for (int r = 0; r < 9; ++r) {
        r_off[r] = o;
        o += r_len[r];
      }
      r_off[9] = o;
    }
    __syncthreads();
    const bool staged = r_off[9] <= CAP;
    if (staged) {
      for (int r = 0; r < 9; ++r)
        for (int t = threadIdx.x; t < r_len[r]; t += kNbrThreads)
          cand[r_off[r] + t] = ld4(spos + r_lo[r] + t);
    }
    __syncthreads();
    for (int p = s0 + w; p < s1; p += nw) {
      const V xi = ld4(spos + p);
      long long base = 0;
      if (FILL) base = row_ptr[svals[p]];
      int cnt = 0;
      for (int r = 0; r < 9; ++r) {
        const int len = r_len[r], lo = r_lo[r], off = r_off[r];
        for (int t0 = 0; t0 < len; t0 += 32) {
          const int t = t0 + lane;
          bool hit = false;
          if (t < len) {
            const V xj = staged ? cand[off + t] : ld4(spos + lo + t);
            hit = in_support(xi, xj);
          }
          const unsigned m = __ballot_sync(0xffffffffu, hit);
          if (FILL && hit) col[base + cnt + __popc(m & lt)] = svals[lo + t];
          cnt += __popc(m);
        }
      }
      if (!FILL && lane == 0) counts[svals[p]] = cnt;
    }
    __syncthreads();
  }
}

__global__ void k_check_nnz(const long long *row_ptr, int64_t n, long long cap_nnz,
                            int64_t *nnz_dev, DevStatus *st, const GridDev *g) {
  if (!g->ok) return;
  long long nnz = row_ptr[n];
  st->nnz = nnz;
  if (nnz_dev) *nnz_dev = nnz;
  if (nnz > cap_nnz) set_error(st, MAFP_ECAPACITY, nnz);
}

// ------------------------------------------------ warp-per-cell mask path
// Every particle of a cell shares the candidate set "27 cells around it",
// which is 9 runs of consecutive sorted positions (3 x-adjacent cells each).
// Each warp takes occupied cells from a device work queue (an atomic ticket
// per cell) and handles its cell alone, with warp-level synchronisation only:
// a film cell (a dozen particles, ~4 candidate words) and a 3D cell (~40
// particles, ~37 words) then cost the warp in proportion to their work, and
// no block waits at a barrier for its slowest thread.  The candidates are
// staged in windows of kWinWords words (32 candidates each) in the warp's part
// of shared memory; the warp's lanes take (word, particle) items of the window
// (consecutive lanes, consecutive particles of one word: the candidate reads
// are broadcasts), test 32 candidates against the particle and write one bit
// per candidate (word-major mask[w * stride + p], coalesced) plus the row
// length.  The fill kernel turns the bits back into column indices, so the
// distance tests run once.
constexpr int kMaskThreads = 128;
constexpr int kMaskWarps = kMaskThreads / 32;
constexpr int kMaskMaxP = 256;   // particles of one cell in the mask kernel (else: overflow path)
static_assert(kMaskCap < 65536 && kMaskMaxP % 2 == 0, "two 16-bit hit counts per word");
// FP32 window: four arrays (x, y, z, h/2) of kWinWords words, two pad floats
// per word: a float2 read gives two consecutive candidates, and the words that
// lanes of one warp test sit in different banks.  FP64: double4 records, one
// pad record per word.
template <typename T> struct MaskWin;
template <> struct MaskWin<float> {
  static constexpr int WORDS = 11;
  static constexpr int SOA = 32 * WORDS + 2 * WORDS;   // floats per array
  static constexpr int TILE_BYTES = 4 * SOA * (int)sizeof(float);
};
template <> struct MaskWin<double> {
  static constexpr int WORDS = 5;
  static constexpr int TILE_BYTES = (32 * WORDS + WORDS) * (int)sizeof(double4_16a);
};
template <typename T>
constexpr int kMaskWarpBytes = MaskWin<T>::TILE_BYTES + (kMaskMaxP / 2) * (int)sizeof(unsigned);

constexpr int kFillThreads = 128;
constexpr int kFillWarps = kFillThreads / 32;
constexpr int kFillWinWords = 16;   // candidate words of one fill window

// Rows of the 27-cell neighbourhood of global cell `key`: run r (dz = r/3-1,
// dy = r%3-1) covers cells key-1..key+1 of that (y, z) row of the key's own
// cloud grid, clipped to that grid.
__device__ __forceinline__ void cell_runs(int key, const CloudGrids &cg,
                                          const int32_t *cell_start, const int32_t *cell_end,
                                          int r, int *lo_out, int *len_out) {
  int b0 = 0, b1 = cg.nb;   // cloud with cell_base[b] <= key < cell_base[b + 1]
  while (b1 - b0 > 1) {
    const int mid = (b0 + b1) >> 1;
    if (cg.cell_base[mid] <= key) b0 = mid; else b1 = mid;
  }
  const GridDev &g = cg.grids[b0];
  const int local = key - (int)cg.cell_base[b0];
  const int dx_ = g.dim[0], dy_ = g.dim[1], dz_ = g.dim[2];
  const int cx = local % dx_, cy = (local / dx_) % dy_, cz = local / (dx_ * dy_);
  const int ddz = r / 3 - 1, ddy = r % 3 - 1;
  int lo = INT_MAX, hi = 0;
  if (cz + ddz >= 0 && cz + ddz < dz_ && cy + ddy >= 0 && cy + ddy < dy_) {
    const int base = key + ddz * dx_ * dy_ + ddy * dx_;
    const int k0 = cx > 0 ? base - 1 : base, k1 = cx < dx_ - 1 ? base + 1 : base;
    for (int k = k0; k <= k1; ++k) {
      lo = min(lo, cell_start[k]);
      hi = max(hi, cell_end[k]);
    }
  }
  *lo_out = lo;
  *len_out = hi > lo ? hi - lo : 0;
}

// The 9 runs of a cell, one per lane 0..8 (start, length, offset in the
// cell's candidate list), and the candidate total (every lane).
__device__ __forceinline__ void warp_cell_runs(int key, const CloudGrids &cg,
                                               const int32_t *cell_start,
                                               const int32_t *cell_end, int lane, int *lo,
                                               int *len, int *off, int *total) {
  *lo = 0;
  *len = 0;
  if (lane < 9) cell_runs(key, cg, cell_start, cell_end, lane, lo, len);
  int inc = *len;
#pragma unroll
  for (int o = 1; o < 16; o <<= 1) {
    const int u = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += u;
  }
  *off = inc - *len;
  *total = __shfl_sync(0xffffffffu, inc, 8);
}

// Calls put(c - c0, sorted position of candidate c) for every candidate c of
// the window [c0, c1), lanes striding over each run's part of the window.
template <typename F>
__device__ __forceinline__ void for_window(int lo, int len, int off, int c0, int c1, int lane,
                                           F &&put) {
#pragma unroll 1
  for (int r = 0; r < 9; ++r) {
    const int rlo = __shfl_sync(0xffffffffu, lo, r), rlen = __shfl_sync(0xffffffffu, len, r);
    const int roff = __shfl_sync(0xffffffffu, off, r);
    const int a = max(c0, roff), b = min(c1, roff + rlen);
    for (int c = a + lane; c < b; c += 32) put(c - c0, rlo + (c - roff));
  }
}

// FP32 test with an explicit band: certainly in / certainly out from FP32,
// the FP64 definition inside +-1e-5 of the bound.
__device__ __forceinline__ bool support_test(const float4 &a, const float4 &b) {
  const float dx = b.x - a.x, dy = b.y - a.y, dz = b.z - a.z;
  const float d2 = (dx * dx + dy * dy) + dz * dz;
  const float r = (a.w + b.w) * 0.5f;
  const float r2 = r * r;
  if (d2 < r2 * 0.99999f) return true;
  if (d2 > r2 * 1.00001f) return false;
  return in_support64(a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w);
}
__device__ __forceinline__ bool support_test(const double4_16a &a, const double4_16a &b) {
  return in_support64(a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w);
}

template <typename T>
__global__ void __launch_bounds__(kMaskThreads) k_nbr_mask(
    CloudGrids cg, const int32_t *ucell, int32_t *n_ucell, const vec4_t<T> *spos,
    const int32_t *svals, const int32_t *cell_start, const int32_t *cell_end, int32_t *counts,
    uint32_t *mask, int64_t stride, int32_t *overflow, int32_t *n_overflow, int64_t n) {
  using V = vec4_t<T>;
  constexpr int WW = MaskWin<T>::WORDS;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
  unsigned char *mine = smem_raw + wp * kMaskWarpBytes<T>;
  V *cand = reinterpret_cast<V *>(mine);
  float *tx = reinterpret_cast<float *>(mine);
  float *ty = tx + (sizeof(T) == 4 ? MaskWin<float>::SOA : 0);
  float *tz = ty + (sizeof(T) == 4 ? MaskWin<float>::SOA : 0);
  float *th = tz + (sizeof(T) == 4 ? MaskWin<float>::SOA : 0);
  // per-particle hit counts, two 16-bit counts per word (a row has at most
  // kMaskCap < 65536 candidates)
  unsigned *cnt = reinterpret_cast<unsigned *>(mine + MaskWin<T>::TILE_BYTES);
  if (!cg.all->ok) return;
  const int nbig = n_ucell[0], nu = nbig + n_ucell[4];
  for (;;) {
    // cells are handed out one at a time (work ticket n_ucell[2]): a warp that
    // finishes a light film cell takes the next cell at once
    int t = 0;
    if (lane == 0) t = atomicAdd(n_ucell + 2, 1);
    t = __shfl_sync(0xffffffffu, t, 0);
    if (t >= nu) break;
    const int cb = cell_slot(t, nbig, n);
    const int key = ucell[2 * cb], s0 = ucell[2 * cb + 1];
    const int P = cell_end[key] - s0;
    int lo, len, off, total;
    warp_cell_runs(key, cg, cell_start, cell_end, lane, &lo, &len, &off, &total);
    if (total > kMaskCap || P > kMaskMaxP) {
      // too many candidates for the mask words, or particles for the counters:
      // the warp-per-particle kernel takes the cell
      if (lane == 0) overflow[atomicAdd(n_overflow, 1)] = cb;
      continue;
    }
    for (int q = lane; q < (P + 1) / 2; q += 32) cnt[q] = 0u;
    const int nwords = (total + 31) >> 5;
    for (int w0 = 0; w0 < nwords; w0 += WW) {
      const int w1 = min(nwords, w0 + WW);
      __syncwarp();   // the previous window's reads are done
      for_window(lo, len, off, w0 * 32, min(total, w1 * 32), lane, [&](int c, int sp) {
        const V v = ld4(spos + sp);
        if constexpr (sizeof(T) == 4) {
          const int sl = c + 2 * (c >> 5);
          tx[sl] = v.x;
          ty[sl] = v.y;
          tz[sl] = v.z;
          th[sl] = 0.5f * v.w;   // exact: r = h_i / 2 + h_j / 2 = (h_i + h_j) / 2
        } else {
          cand[c + (c >> 5)] = v;
        }
      });
      __syncwarp();
      // one work item = (word, particle); consecutive lanes take consecutive
      // particles of a word, so small cells still fill the warp
      const int items = P * (w1 - w0);
      for (int it = lane; it < items; it += 32) {
        const int wl = it / P, q = it - wl * P;
        const int w = w0 + wl;
        const int base = w << 5;
        const uint32_t valid = (total - base) >= 32 ? 0xffffffffu : ((1u << (total - base)) - 1u);
        const V xi = ld4(spos + s0 + q);
        uint32_t m = 0, band = 0;
        if constexpr (sizeof(T) == 4) {
          // two candidates per packed FP32 instruction; the window always
          // holds 32 * WW slots (plus pads), so reads past `total` stay in it
          // and are masked off
          const float hi2 = 0.5f * xi.w;
          const float2 nx = make_float2(-xi.x, -xi.x), ny = make_float2(-xi.y, -xi.y);
          const float2 nz = make_float2(-xi.z, -xi.z), hh = make_float2(hi2, hi2);
          const float2 klo = make_float2(0.99999f, 0.99999f), khi = make_float2(1.00001f, 1.00001f);
          const int sb = 34 * wl;   // slot of candidate 32 w in the window
#pragma unroll
          for (int k = 0; k < 32; k += 2) {
            const float2 bx = *reinterpret_cast<const float2 *>(tx + sb + k);
            const float2 by = *reinterpret_cast<const float2 *>(ty + sb + k);
            const float2 bz = *reinterpret_cast<const float2 *>(tz + sb + k);
            const float2 bh = *reinterpret_cast<const float2 *>(th + sb + k);
            const float2 dx = __fadd2_rn(bx, nx), dy = __fadd2_rn(by, ny), dz = __fadd2_rn(bz, nz);
            float2 d2 = __fmul2_rn(dx, dx);
            d2 = __ffma2_rn(dy, dy, d2);
            d2 = __ffma2_rn(dz, dz, d2);
            const float2 r = __fadd2_rn(bh, hh);
            const float2 r2 = __fmul2_rn(r, r);
            const float2 l2 = __fmul2_rn(r2, klo), h2 = __fmul2_rn(r2, khi);
            m |= (d2.x < l2.x ? 1u : 0u) << k;
            m |= (d2.y < l2.y ? 1u : 0u) << (k + 1);
            band |= (d2.x <= h2.x ? 1u : 0u) << k;
            band |= (d2.y <= h2.y ? 1u : 0u) << (k + 1);
          }
          m &= valid;
          band &= valid & ~m;
          // pairs within 1e-5 of the bound: the FP64 definition decides
          while (band) {
            const int k = __ffs(band) - 1;
            band &= band - 1;
            const int sl = sb + k;
            if (in_support64(xi.x, xi.y, xi.z, xi.w, tx[sl], ty[sl], tz[sl], 2.0f * th[sl]))
              m |= 1u << k;
          }
        } else {
          const V *cw = cand + 33 * wl;   // slot of candidate 32 w in the window
          for (int k = 0; k < 32; ++k)
            if ((valid >> k) & 1u)
              if (support_test(xi, cw[k])) m |= 1u << k;
        }
        mask[(int64_t)w * stride + s0 + q] = m;
        atomicAdd(&cnt[q >> 1], (unsigned)__popc(m) << ((q & 1) * 16));
      }
    }
    __syncwarp();
    for (int q = lane; q < P; q += 32)
      counts[svals[s0 + q]] = (int)((cnt[q >> 1] >> ((q & 1) * 16)) & 0xffffu);
    __syncwarp();   // the counters are read before the next cell clears them
  }
}

// Fill pass for the mask kernel's cells, also one warp per cell from a work
// queue.  The cell's particles go in chunks of 32 (lane = particle, its row
// start and running length in registers); for each window of kFillWinWords
// candidate words the warp stages the candidates' original indices and the
// chunk's hit words (coalesced) in its part of shared memory, then expands the
// chunk's rows one particle at a time: one candidate per lane, ballot-free
// compaction by popcount into the row, coalesced stores.  Rows come out
// ascending when the cloud is in cell order (candidates are runs of
// consecutive sorted positions, ascending).
__global__ void __launch_bounds__(kFillThreads) k_nbr_fill(
    CloudGrids cg, const int32_t *ucell, int32_t *n_ucell, const int32_t *svals,
    const int32_t *cell_start, const int32_t *cell_end, const uint32_t *mask, int64_t stride,
    const long long *row_ptr, int32_t *col, long long cap_nnz, int64_t n) {
  __shared__ int32_t cand_v[kFillWarps][kFillWinWords * 32];   // original indices
  __shared__ uint32_t mw[kFillWarps][kFillWinWords][32];       // hit words of the chunk
  if (!cg.all->ok) return;
  if (row_ptr[n] > cap_nnz) return;
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
  const unsigned lt = (1u << lane) - 1u;
  int32_t *cv = cand_v[wp];
  const int nbig = n_ucell[0], nu = nbig + n_ucell[4];
  for (;;) {
    int t = 0;
    if (lane == 0) t = atomicAdd(n_ucell + 3, 1);   // work ticket, as in the mask kernel
    t = __shfl_sync(0xffffffffu, t, 0);
    if (t >= nu) break;
    const int cb = cell_slot(t, nbig, n);
    const int key = ucell[2 * cb], s0 = ucell[2 * cb + 1];
    const int P = cell_end[key] - s0;
    int lo, len, off, total;
    warp_cell_runs(key, cg, cell_start, cell_end, lane, &lo, &len, &off, &total);
    if (total > kMaskCap || P > kMaskMaxP) continue;   // the overflow path fills it
    const int nwords = (total + 31) >> 5;
    for (int p0 = 0; p0 < P; p0 += 32) {
      const int np = min(32, P - p0);
      const int q = p0 + lane;
      const long long rs = lane < np ? row_ptr[svals[s0 + q]] : 0;
      int at = 0;
      for (int w0 = 0; w0 < nwords; w0 += kFillWinWords) {
        const int w1 = min(nwords, w0 + kFillWinWords);
        __syncwarp();   // the previous window's reads are done
        for_window(lo, len, off, w0 * 32, min(total, w1 * 32), lane,
                   [&](int c, int sp) { cv[c] = svals[sp]; });
        for (int w = w0; w < w1; ++w)
          mw[wp][w - w0][lane] = lane < np ? mask[(int64_t)w * stride + s0 + q] : 0u;
        __syncwarp();
        // this lane's candidate of every word of the window, in registers (the
        // window loop is unrolled; words past w1 are empty)
        int32_t cvr[kFillWinWords];
#pragma unroll
        for (int ww = 0; ww < kFillWinWords; ++ww)
          cvr[ww] = w0 + ww < w1 ? cv[ww * 32 + lane] : 0;
        for (int k = 0; k < np; ++k) {
          int32_t *crow = col + __shfl_sync(0xffffffffu, rs, k);
          int a = __shfl_sync(0xffffffffu, at, k);
#pragma unroll
          for (int ww = 0; ww < kFillWinWords; ++ww) {
            const uint32_t word = w0 + ww < w1 ? mw[wp][ww][k] : 0u;
            if ((word >> lane) & 1u) crow[a + __popc(word & lt)] = cvr[ww];
            a += __popc(word);
          }
          if (lane == k) at = a;
        }
      }
    }
  }
}

// Rows come out ascending in cell order; when the input order differs from the
// cell order each row is sorted (bitonic, one warp per row, in shared memory).
constexpr int kSortWarps = 4;

__global__ void __launch_bounds__(kSortWarps * 32) k_rowsort(const long long *row_ptr,
                                                             int32_t *col, int64_t n,
                                                             long long cap_nnz,
                                                             DevStatus *st, const GridDev *g) {
  if (!g->ok || !st->not_identity) return;
  if (row_ptr[n] > cap_nnz) return;
  __shared__ int32_t buf[kSortWarps][kMaxRowSort];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int32_t *a = buf[w];
  for (int64_t i = (int64_t)blockIdx.x * kSortWarps + w; i < n;
       i += (int64_t)gridDim.x * kSortWarps) {
    const long long b = row_ptr[i];
    const int len = (int)(row_ptr[i + 1] - b);
    if (len > kMaxRowSort) {
      if (lane == 0) set_error(st, MAFP_ECAPACITY, len);
      continue;
    }
    int P = 1;
    while (P < len) P <<= 1;
    for (int t = lane; t < P; t += 32) a[t] = t < len ? col[b + t] : INT_MAX;
    __syncwarp();
    for (int k = 2; k <= P; k <<= 1)
      for (int j = k >> 1; j > 0; j >>= 1) {
        for (int t = lane; t < P; t += 32) {
          int u = t ^ j;
          if (u > t) {
            int x = a[t], y = a[u];
            bool asc = (t & k) == 0;
            if ((x > y) == asc) {
              a[t] = y;
              a[u] = x;
            }
          }
        }
        __syncwarp();
      }
    for (int t = lane; t < len; t += 32) col[b + t] = a[t];
    __syncwarp();
  }
}

// tloc[e] = position of i inside row j for the entry e = (i, j).
__global__ void k_tmap(const long long *row_ptr, const int32_t *col, int64_t n, uint16_t *tloc,
                       DevStatus *st) {
  const int lane = threadIdx.x & 31;
  const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i = wid; i < n; i += nwarps) {
    const long long b = row_ptr[i], e1 = row_ptr[i + 1];
    for (long long e = b + lane; e < e1; e += 32) {
      const int j = col[e];
      long long lo = row_ptr[j], hi = row_ptr[j + 1];
      const long long rb = lo;
      if (hi - rb > 65535) {
        set_error(st, MAFP_ECAPACITY, hi - rb);
        continue;
      }
      while (lo < hi) {
        long long mid = (lo + hi) >> 1;
        if (col[mid] < i) lo = mid + 1; else hi = mid;
      }
      tloc[e] = (uint16_t)(lo - rb);
    }
  }
}

// ------------------------------------------------------------------ host side
// A1: grids, cell keys, stable radix sort, cell ranges, sorted positions and
// (optionally) the cell order.  On return the sorted keys / indices are in
// *kin / *vin.
template <typename T>
static int sort_into_cells_t(mafp_ctx *ctx, int64_t n, int nb, const long long *cloud_off,
                             const void *pos_h, int32_t *order, uint32_t **kin_out,
                             int32_t **vin_out, cudaStream_t s) {
  using V = vec4_t<T>;
  const V *pos = reinterpret_cast<const V *>(pos_h);
  const int sms = sm_count();
  const int parts = std::max(1, std::min(kBoxBlocks / std::max(nb, 1), kBoxPartsMax));
  MAFP_TIMED(ctx, s, "k_cloud_bbox",
             k_cloud_bbox<T><<<nb * parts, kBoxThreads, 0, s>>>(pos, n, cloud_off, nb, parts,
                                                                 ctx->cloud_partial,
                                                                 ctx->cloud_id));
  MAFP_TIMED(ctx, s, "k_cloud_fold",
             k_cloud_fold<<<(nb + kBoxThreads / 32 - 1) / (kBoxThreads / 32), kBoxThreads, 0, s>>>(
                 ctx->cloud_partial, nb, parts));
  MAFP_TIMED(ctx, s, "k_cloud_grid",
             k_cloud_grid<<<1, kBoxThreads, 0, s>>>(ctx->cloud_partial, cloud_off, n, nb, parts,
                                                    ctx->d_grids,
                                                    ctx->cell_base, ctx->d_grid, ctx->d_status,
                                                    ctx->cap_cells,
                                                    0.01 * (double)ctx->tune.cell_edge_pct));
  CloudGrids cg{ctx->d_grids, ctx->cell_base, nb, ctx->d_grid};
  MAFP_TIMED(ctx, s, "k_hash",
             k_hash<T><<<grid_for(n, 256, sms * 16), 256, 0, s>>>(pos, n, ctx->cloud_id, cg,
                                                                  ctx->keys_a, ctx->vals_a));
  MAFP_TIMED(ctx, s, "k_clear_cells",
             k_clear_cells<<<sms * 8, 256, 0, s>>>(ctx->d_grid, ctx->cell_start, ctx->cell_end,
                                                   ctx->n_ucell));
  MAFP_LAUNCH_CHECK(ctx);
  const int tiles = (int)((n + kRadixTile - 1) / kRadixTile);
  uint32_t *kin = ctx->keys_a, *kout = ctx->keys_b;
  int32_t *vin = ctx->vals_a, *vout = ctx->vals_b;
  long long *offs = reinterpret_cast<long long *>(ctx->remap_i64);
  for (int p = 0; p < ctx->radix_passes; ++p) {
    MAFP_TIMED(ctx, s, "k_radix_hist",
               k_radix_hist<<<tiles, kRadixThreads, 0, s>>>(kin, n, 8 * p, ctx->radix_hist, tiles,
                                                  ctx->d_grid));
    int rc = scan_i32_to_i64(ctx, ctx->radix_hist, offs, (int64_t)256 * tiles, s);
    if (rc) return rc;
    MAFP_TIMED(ctx, s, "k_radix_scatter",
               k_radix_scatter<<<tiles, kRadixThreads, 0, s>>>(kin, vin, kout, vout, n, 8 * p, offs, tiles,
                                                     ctx->d_grid));
    MAFP_LAUNCH_CHECK(ctx);
    uint32_t *tk = kin; kin = kout; kout = tk;
    int32_t *tv = vin; vin = vout; vout = tv;
  }
  V *spos = reinterpret_cast<V *>(ctx->spos);
  MAFP_TIMED(ctx, s, "k_cells<T>",
             k_cells<T><<<grid_for(n, 256, sms * 16), 256, 0, s>>>(kin, vin, n, pos, spos, ctx->cell_start,
                                                        ctx->cell_end, ctx->ucell, ctx->n_ucell,
                                                        ctx->d_status, order, ctx->d_grid));
  MAFP_TIMED(ctx, s, "k_identity_flag",
             k_identity_flag<<<1, 1, 0, s>>>(ctx->d_status));
  MAFP_LAUNCH_CHECK(ctx);
  *kin_out = kin;
  *vin_out = vin;
  return MAFP_OK;
}

template <typename T>
static int build_neighbours_t(mafp_ctx *ctx, int64_t n, int nb, const long long *cloud_off,
                              const void *pos_h, int64_t *row_ptr, int32_t *col,
                              int64_t cap_nnz, int64_t *nnz_dev, int32_t *order, cudaStream_t s) {
  using V = vec4_t<T>;
  const int sms = sm_count();
  uint32_t *kin = nullptr;
  int32_t *vin = nullptr;
  int rc0 = sort_into_cells_t<T>(ctx, n, nb, cloud_off, pos_h, order, &kin, &vin, s);
  if (rc0) return rc0;
  V *spos = reinterpret_cast<V *>(ctx->spos);
  CloudGrids cg{ctx->d_grids, ctx->cell_base, nb, ctx->d_grid};
  const int nbr_blocks = sms * 8;
  int32_t *n_overflow = ctx->n_ucell + 1;
  const int64_t stride = ctx->cap_particles;
  MAFP_TIMED(ctx, s, sizeof(T) == 4 ? "k_nbr_mask<float>" : "k_nbr_mask<double>",
             k_nbr_mask<T><<<sms * 16, kMaskThreads, kMaskWarps * kMaskWarpBytes<T>, s>>>(
                 cg, ctx->ucell, ctx->n_ucell, spos, vin, ctx->cell_start,
                 ctx->cell_end, ctx->counts, ctx->nbr_mask, stride, ctx->overflow, n_overflow,
                 n));
  MAFP_TIMED(ctx, s, "k_nbr<T,false>(overflow cells)",
             k_nbr<T, false><<<nbr_blocks, kNbrThreads, kNbrSmemBytes, s>>>(
      cg, ctx->ucell, ctx->overflow, n_overflow, spos, vin, ctx->cell_start,
      ctx->cell_end, ctx->counts, nullptr, nullptr, 0, n));
  MAFP_LAUNCH_CHECK(ctx);
  int rc = scan_i32_to_i64(ctx, ctx->counts, reinterpret_cast<long long *>(row_ptr), n, s);
  if (rc) return rc;
  MAFP_TIMED(ctx, s, "k_check_nnz",
             k_check_nnz<<<1, 1, 0, s>>>(reinterpret_cast<const long long *>(row_ptr), n, cap_nnz, nnz_dev,
                              ctx->d_status, ctx->d_grid));
  MAFP_TIMED(ctx, s, "k_nbr_fill",
             k_nbr_fill<<<sms * (2048 / kFillThreads), kFillThreads, 0, s>>>(
                 cg, ctx->ucell, ctx->n_ucell, vin, ctx->cell_start, ctx->cell_end,
                 ctx->nbr_mask, stride, reinterpret_cast<const long long *>(row_ptr), col,
                 cap_nnz, n));
  MAFP_TIMED(ctx, s, "k_nbr<T,true>(overflow cells)",
             k_nbr<T, true><<<nbr_blocks, kNbrThreads, kNbrSmemBytes, s>>>(
      cg, ctx->ucell, ctx->overflow, n_overflow, spos, vin, ctx->cell_start,
      ctx->cell_end, ctx->counts, reinterpret_cast<const long long *>(row_ptr), col, cap_nnz, n));
  MAFP_TIMED(ctx, s, "k_rowsort",
             k_rowsort<<<grid_for(n, kSortWarps, sms * 8), kSortWarps * 32, 0, s>>>(
      reinterpret_cast<const long long *>(row_ptr), col, n, cap_nnz, ctx->d_status,
      ctx->d_grid));
  MAFP_LAUNCH_CHECK(ctx);
  return MAFP_OK;
}

int build_neighbours(mafp_ctx *ctx, int64_t n, int32_t dtype, const void *pos_h,
                     int64_t *row_ptr, int32_t *col, int64_t cap_nnz, int64_t *nnz_dev,
                     int32_t *order, cudaStream_t s) {
  MAFP_TIMED(ctx, s, "k_set_one_cloud", k_set_one_cloud<<<1, 1, 0, s>>>(ctx->one_cloud, n));
  if (dtype == MAFP_F64)
    return build_neighbours_t<double>(ctx, n, 1, ctx->one_cloud, pos_h, row_ptr, col, cap_nnz,
                                      nnz_dev, order, s);
  return build_neighbours_t<float>(ctx, n, 1, ctx->one_cloud, pos_h, row_ptr, col, cap_nnz,
                                   nnz_dev, order, s);
}

int cell_order(mafp_ctx *ctx, int64_t n, int32_t dtype, const void *pos_h, int32_t *order,
               cudaStream_t s) {
  MAFP_TIMED(ctx, s, "k_set_one_cloud", k_set_one_cloud<<<1, 1, 0, s>>>(ctx->one_cloud, n));
  uint32_t *kin = nullptr;
  int32_t *vin = nullptr;
  if (dtype == MAFP_F64)
    return sort_into_cells_t<double>(ctx, n, 1, ctx->one_cloud, pos_h, order, &kin, &vin, s);
  return sort_into_cells_t<float>(ctx, n, 1, ctx->one_cloud, pos_h, order, &kin, &vin, s);
}

int build_neighbours_batched(mafp_ctx *ctx, int64_t n, int32_t dtype, int32_t nclouds,
                             const int64_t *cloud_offset, const void *pos_h, int64_t *row_ptr,
                             int32_t *col, int64_t cap_nnz, int64_t *nnz_dev, int32_t *order,
                             cudaStream_t s) {
  const long long *off = reinterpret_cast<const long long *>(cloud_offset);
  if (dtype == MAFP_F64)
    return build_neighbours_t<double>(ctx, n, nclouds, off, pos_h, row_ptr, col, cap_nnz,
                                      nnz_dev, order, s);
  return build_neighbours_t<float>(ctx, n, nclouds, off, pos_h, row_ptr, col, cap_nnz, nnz_dev,
                                   order, s);
}

void init_kernel_attributes() {
  cudaFuncSetAttribute(k_nbr_mask<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       kMaskWarps * kMaskWarpBytes<float>);
  cudaFuncSetAttribute(k_nbr_mask<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       kMaskWarps * kMaskWarpBytes<double>);
  cudaFuncSetAttribute(k_nbr<float, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       kNbrSmemBytes);
  cudaFuncSetAttribute(k_nbr<float, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       kNbrSmemBytes);
  cudaFuncSetAttribute(k_nbr<double, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       kNbrSmemBytes);
  cudaFuncSetAttribute(k_nbr<double, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       kNbrSmemBytes);
}

int transpose_map(mafp_ctx *ctx, int64_t n, const int64_t *row_ptr, const int32_t *col,
                  uint16_t *tloc, cudaStream_t s) {
  MAFP_TIMED(ctx, s, "k_tmap",
             k_tmap<<<grid_for(n * 32, 256, sm_count() * 16), 256, 0, s>>>(
      reinterpret_cast<const long long *>(row_ptr), col, n, tloc, ctx->d_status));
  MAFP_LAUNCH_CHECK(ctx);
  return MAFP_OK;
}

}  // namespace mafp
