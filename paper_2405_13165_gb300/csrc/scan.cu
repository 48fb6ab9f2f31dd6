// scan.cu -- device-wide exclusive prefix sum (int32 -> int64), three kernels:
// tile reduce, scan of tile sums (one block), tile down-sweep.
#include "internal.cuh"

namespace mafp {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 16;
constexpr int kScanTile = kScanThreads * kScanItems;  // 4096

template <typename T>
__device__ __forceinline__ T warp_inclusive(T v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    T u = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += u;
  }
  return v;
}

// Exclusive scan of one value per thread across the block; returns the
// thread's exclusive prefix, *total gets the block total.
template <typename T>
__device__ __forceinline__ T block_exclusive(T v, T *total) {
  // [0, 32): per-warp totals, then per-warp exclusive offsets; [32]: block total
  // (a slot of its own: with 32 warps, [31] is the last warp's offset)
  __shared__ T warp_tot[33];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  T inc = warp_inclusive(v);
  if (lane == 31) warp_tot[w] = inc;
  __syncthreads();
  if (w == 0) {
    T t = lane < nw ? warp_tot[lane] : T(0);
    T ti = warp_inclusive(t);
    if (lane < nw) warp_tot[lane] = ti - t;
    if (lane == nw - 1) warp_tot[32] = ti;
  }
  __syncthreads();
  T res = warp_tot[w] + inc - v;
  *total = warp_tot[32];
  __syncthreads();
  return res;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_reduce(const int32_t *in, int64_t n,
                                                              long long *tile_sum) {
  const int64_t base = (int64_t)blockIdx.x * kScanTile;
  long long s = 0;
  for (int k = threadIdx.x; k < kScanTile; k += kScanThreads) {
    int64_t idx = base + k;
    if (idx < n) s += in[idx];
  }
  __shared__ long long red[kScanThreads / 32];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    long long t = 0;
    for (int w = 0; w < kScanThreads / 32; ++w) t += red[w];
    tile_sum[blockIdx.x] = t;
  }
}

// One block scans the tile sums in place (exclusive) and stores the total at [ntiles].
__global__ void __launch_bounds__(1024) k_scan_tiles(long long *tile_sum, int64_t ntiles) {
  long long carry = 0;
  for (int64_t base = 0; base < ntiles; base += 1024) {
    int64_t idx = base + threadIdx.x;
    long long v = idx < ntiles ? tile_sum[idx] : 0;
    long long tot;
    long long ex = block_exclusive<long long>(v, &tot);
    if (idx < ntiles) tile_sum[idx] = carry + ex;
    carry += tot;
  }
  if (threadIdx.x == 0) tile_sum[ntiles] = carry;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_down(const int32_t *in, int64_t n,
                                                            const long long *tile_sum,
                                                            long long *out) {
  const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
  int32_t v[kScanItems];
  long long s = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    int64_t idx = base + k;
    v[k] = idx < n ? in[idx] : 0;
    s += v[k];
  }
  long long tot;
  long long ex = block_exclusive<long long>(s, &tot) + tile_sum[blockIdx.x];
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    int64_t idx = base + k;
    if (idx < n) out[idx] = ex;
    ex += v[k];
  }
  if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) {
    int64_t ntiles = gridDim.x;
    out[n] = tile_sum[ntiles];
  }
}

int scan_i32_to_i64(mafp_ctx *ctx, const int32_t *in, long long *out, int64_t n, cudaStream_t s) {
  if (n <= 0) {
    MAFP_CUDA_TRY(ctx, cudaMemsetAsync(out, 0, sizeof(long long), s));
    return MAFP_OK;
  }
  int64_t ntiles = (n + kScanTile - 1) / kScanTile;
  MAFP_TIMED(ctx, s, "k_scan_reduce",
             k_scan_reduce<<<(unsigned)ntiles, kScanThreads, 0, s>>>(in, n, ctx->scan_tmp));
  MAFP_TIMED(ctx, s, "k_scan_tiles",
             k_scan_tiles<<<1, 1024, 0, s>>>(ctx->scan_tmp, ntiles));
  MAFP_TIMED(ctx, s, "k_scan_down",
             k_scan_down<<<(unsigned)ntiles, kScanThreads, 0, s>>>(in, n, ctx->scan_tmp, out));
  MAFP_LAUNCH_CHECK(ctx);
  return MAFP_OK;
}

}  // namespace mafp
