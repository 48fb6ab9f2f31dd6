// internal.cuh -- shared device helpers and the context layout of libmafp.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>

#include "mafp.h"

namespace mafp {

constexpr int kMaxRowSort = 2048;   // longest row the in-shared-memory row sort handles
constexpr int kMaskCap = 1536;      // candidates of one cell tile in the neighbour mask kernel
constexpr int kMaskWords = kMaskCap / 32;
constexpr int kMaxClouds = 65536;   // clouds of one batched neighbour build

// Device status block (layout mirrored by mafp_status in the public header).
struct DevStatus {
  int32_t code;
  int32_t cells_identity;
  long long required;
  long long nnz;
  long long n_fp64_stencil;
  long long n_fp64_eigen;
  long long n_deficient;
  long long n_near;
  long long n_out;
  long long n_nonfinite;
  long long ncells;
  double cell_size;
  // internal (not copied to the caller)
  int32_t not_identity;
  int32_t fallback_count;
  long long remap_scratch[4];
};

// Neighbour grid, computed on the device from the cloud's bounding box.
struct GridDev {
  double lo[3];
  double c;        // cell edge (>= max h, enlarged when the box would need too many cells)
  double inv_c;
  int32_t dim[3];
  int32_t ok;
  long long ncells;
  double hmax;
};

}  // namespace mafp

struct mafp_ctx {
  mafp_params prm;
  mafp_tuning tune;
  int64_t cap_particles;
  int64_t cap_cells;
  int device;
  int radix_passes;
  int64_t max_tiles;
  // device scratch (all allocated at creation)
  uint32_t *keys_a, *keys_b;
  int32_t *vals_a, *vals_b;
  int32_t *radix_hist;      // [256 * max_tiles] (+1 for the scan total)
  int32_t *cell_start, *cell_end;
  void *spos;               // sorted positions, 32 bytes per particle
  int32_t *ucell;           // [2 * cap] occupied cells: key, first sorted position
  int32_t *n_ucell;         // device counters: cells (front group), overflow cells, mask and
                            // fill tickets, cells (back group)
  int32_t *counts;          // [cap] row lengths
  uint32_t *nbr_mask;       // [kMaskWords * cap] candidate hit bits, word-major
  int32_t *overflow;        // [cap] occupied cells whose candidates overflow the tile
  long long *scan_tmp;      // tile states of the one-pass scan, zero between scans
  int32_t *scan_ctr;        // [2] tickets and finished tiles of the scan, zero between scans
  int32_t *fallback;        // [cap] particles re-done in FP64
  mafp::DevStatus *d_status;
  mafp::GridDev *d_grid;     // all-clouds flag and totals
  mafp::GridDev *d_grids;    // [kMaxClouds] one grid per cloud
  long long *cell_base;      // [kMaxClouds + 1] first global cell of each cloud
  int32_t *cloud_id;         // [cap] cloud of every particle
  long long *one_cloud;      // [2] offsets of the single-cloud case
  double *cloud_partial;     // [(kMaxClouds + 16384) * 8] bounding-box partials
  int64_t *remap_i64;       // [3 * cap + 8]
  int32_t *remap_i32;       // [2 * cap]
  char err[512];
  // kernel-level CUDA-event timing (off unless mafp_profile(ctx, 1))
  int prof_on;
  int prof_n;
  cudaEvent_t *prof_ev;     // 2 * kProfCap events
  const char **prof_name;   // kProfCap names
};

namespace mafp {

#define MAFP_CUDA_TRY(ctx, expr)                                                    \
  do {                                                                              \
    cudaError_t e_ = (expr);                                                        \
    if (e_ != cudaSuccess) {                                                        \
      snprintf((ctx)->err, sizeof((ctx)->err), "%s: %s (%s:%d)", #expr,             \
               cudaGetErrorString(e_), __FILE__, __LINE__);                         \
      return MAFP_ECUDA;                                                            \
    }                                                                               \
  } while (0)

#define MAFP_LAUNCH_CHECK(ctx)                                                      \
  do {                                                                              \
    cudaError_t e_ = cudaGetLastError();                                            \
    if (e_ != cudaSuccess) {                                                        \
      snprintf((ctx)->err, sizeof((ctx)->err), "launch: %s (%s:%d)",                \
               cudaGetErrorString(e_), __FILE__, __LINE__);                         \
      return MAFP_ECUDA;                                                            \
    }                                                                               \
  } while (0)

__device__ inline void set_error(DevStatus *st, int code, long long required) {
  if (atomicCAS(&st->code, 0, code) == 0) st->required = required;
}

// Real-type traits: x4 vector of the storage type.
template <typename T> struct Vec4;
template <> struct Vec4<float> { using type = float4; };
template <> struct Vec4<double> { using type = double4_16a; };
template <typename T> using vec4_t = typename Vec4<T>::type;

__device__ __forceinline__ float4 ld4(const float4 *p) { return __ldg(p); }
__device__ __forceinline__ double4_16a ld4(const double4_16a *p) {
  const double2 *q = reinterpret_cast<const double2 *>(p);
  double2 a = __ldg(q), b = __ldg(q + 1);
  return make_double4_16a(a.x, a.y, b.x, b.y);
}
__device__ __forceinline__ void st4(float4 *p, float4 v) { *p = v; }
__device__ __forceinline__ void st4(double4_16a *p, double4_16a v) {
  double2 *q = reinterpret_cast<double2 *>(p);
  q[0] = make_double2(v.x, v.y);
  q[1] = make_double2(v.z, v.w);
}
template <typename T> __device__ __forceinline__ vec4_t<T> mk4(T a, T b, T c, T d);
template <> __device__ __forceinline__ float4 mk4<float>(float a, float b, float c, float d) {
  return make_float4(a, b, c, d);
}
template <> __device__ __forceinline__ double4_16a mk4<double>(double a, double b, double c, double d) {
  return make_double4_16a(a, b, c, d);
}

// Lanes of the aligned group of G consecutive lanes (G a power of two <= 32)
// that contains the calling thread.  Groups of one warp may diverge: every
// collective below names only its own group's lanes.
template <int G>
__device__ __forceinline__ unsigned group_mask() {
  if constexpr (G == 32) {
    return 0xffffffffu;
  } else {
    return ((1u << G) - 1u) << ((threadIdx.x & 31) & ~(G - 1));
  }
}

// Sum over the group.
template <int G, typename T>
__device__ __forceinline__ T group_sum(T v) {
  const unsigned m = group_mask<G>();
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) v += __shfl_xor_sync(m, v, o, G);
  return v;
}

template <int G>
__device__ __forceinline__ int group_any(int v) {
  const unsigned m = group_mask<G>();
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) v |= __shfl_xor_sync(m, v, o, G);
  return v;
}

// Reduce-scatter of V values over a group of G lanes: on return lane l of the
// group holds in a[0 .. V/G) the group sums of entries l*(V/G) .. l*(V/G)+V/G-1.
// V must be a multiple of G.  Cost: V/2 + V/4 + ... + V/G shuffles.
template <int G, int V, typename T>
__device__ __forceinline__ void reduce_scatter(T (&a)[V]) {
  const int lane = threadIdx.x & (G - 1);
  const unsigned m = group_mask<G>();
#pragma unroll
  for (int o = G / 2, H = V / 2; o > 0; o >>= 1, H >>= 1) {
    const bool up = (lane & o) != 0;
#pragma unroll
    for (int k = 0; k < H; ++k) {
      T send = up ? a[k] : a[k + H];
      T keep = up ? a[k + H] : a[k];
      a[k] = keep + __shfl_xor_sync(m, send, o, G);
    }
  }
}

__device__ __forceinline__ void inc_ll(long long *p, long long v = 1) {
  atomicAdd(reinterpret_cast<unsigned long long *>(p), (unsigned long long)v);
}

template <typename T> __device__ __forceinline__ bool finite_(T x) { return isfinite(x); }

// Launch helpers
inline int grid_for(int64_t work, int per_block, int max_blocks = 1 << 20) {
  int64_t b = (work + per_block - 1) / per_block;
  if (b < 1) b = 1;
  if (b > max_blocks) b = max_blocks;
  return (int)b;
}

int sm_count();

// Launch shapes of a new context (and of the context-free entry point).
inline void default_tuning(mafp_tuning *t) {
  t->stencil3d_group = 32;
  t->stencil2d_group = 8;
  t->apply_group = 8;
  t->grad3d_group = 2;
  t->grad2d_group = 2;
  t->cell_edge_pct = 100;
  t->classify_group = 2;
}

// Name of a kernel instance for the timing record: built once (function-local
// statics are initialised thread-safely) and never written again, so launches
// from several host threads or devices share it safely.
struct KernelName {
  char s[96];
  template <typename... A>
  explicit KernelName(const char *fmt, A... a) {
    snprintf(s, sizeof(s), fmt, a...);
  }
};

// One bit per device (devices 0..63): set once a per-device, per-function
// setting (such as a dynamic shared-memory limit) has been applied there.
// Returns true when the caller still has to apply it on `dev`.
inline bool first_on_device(unsigned long long *mask, int dev) {
  if (dev < 0 || dev >= 64) return true;
  const unsigned long long bit = 1ull << dev;
  return (__atomic_fetch_or(mask, bit, __ATOMIC_ACQ_REL) & bit) == 0;
}

constexpr int kProfCap = 4096;

// Bracket one kernel launch with CUDA events on its stream when profiling is on.
inline void prof_begin(mafp_ctx *ctx, cudaStream_t s) {
  if (ctx->prof_on && ctx->prof_n < kProfCap) cudaEventRecord(ctx->prof_ev[2 * ctx->prof_n], s);
}
inline void prof_end(mafp_ctx *ctx, cudaStream_t s, const char *name) {
  if (ctx->prof_on && ctx->prof_n < kProfCap) {
    cudaEventRecord(ctx->prof_ev[2 * ctx->prof_n + 1], s);
    ctx->prof_name[ctx->prof_n++] = name;
  }
}
#define MAFP_TIMED(ctx, s, name, ...) \
  do {                                \
    prof_begin(ctx, s);               \
    __VA_ARGS__;                      \
    prof_end(ctx, s, name);           \
  } while (0)

// Device-wide exclusive scan of int32 values into int64 prefix (out[n] = total).
int scan_i32_to_i64(mafp_ctx *ctx, const int32_t *in, long long *out, int64_t n,
                    cudaStream_t s);

}  // namespace mafp
