// scan.cu -- device-wide exclusive prefix sum (int32 -> int64) in one pass:
// decoupled look-back over tiles of 4096 values (Merrill and Garland, "Single-
// pass parallel prefix scan with decoupled look-back", 2016).  Each block
// takes the next tile by ticket, publishes its tile sum, walks back over the
// tiles before it until it meets one that has published its inclusive prefix,
// publishes its own and writes its values.  A block only waits on tiles whose
// blocks took their tickets earlier (so they are running or done); every wait
// is bounded (params.wait_limit polls).  A block whose wait runs out records
// MAFP_ETIMEOUT in the status block and computes its prefix itself, summing
// every value before its tile, so the outputs stay exact (consumers of a scan,
// e.g. the radix sort's scatter, index memory with them).  The last block to
// finish clears the tile states and tickets for the next scan, so no reset is
// launched (and a replayed CUDA graph stays valid).
#include "internal.cuh"

namespace mafp {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 16;
constexpr int kScanTile = kScanThreads * kScanItems;  // 4096

// tile state word: flag in bits 62-63 (0 none, 1 tile sum, 2 inclusive prefix),
// value (non-negative) in bits 0-61
constexpr unsigned long long kFlagSum = 1ull << 62, kFlagIncl = 2ull << 62;
constexpr unsigned long long kValueMask = (1ull << 62) - 1;

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

__device__ __forceinline__ unsigned long long load_state(const unsigned long long *p) {
  return *reinterpret_cast<const volatile unsigned long long *>(p);
}
__device__ __forceinline__ void store_state(unsigned long long *p, unsigned long long v) {
  *reinterpret_cast<volatile unsigned long long *>(p) = v;
}

__global__ void __launch_bounds__(kScanThreads) k_scan(const int32_t *in, long long *out,
                                                       int64_t n, int ntiles,
                                                       unsigned long long *state, int *ctr,
                                                       DevStatus *st, long long wait_limit) {
  __shared__ int s_tile, s_last, s_gave_up;
  __shared__ long long s_prefix, s_red[kScanThreads / 32];
  if (threadIdx.x == 0) s_tile = atomicAdd(ctr, 1);
  __syncthreads();
  const int tile = s_tile;
  if (tile >= ntiles) {
    // a ticket beyond this scan's tiles: only possible when two calls of one
    // context overlap on the GPU, which the interface rules out; touch nothing
    if (threadIdx.x == 0) set_error(st, MAFP_EINVAL, tile);
    return;
  }
  const int64_t base = (int64_t)tile * kScanTile + (int64_t)threadIdx.x * kScanItems;
  int32_t v[kScanItems];
  long long s = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    const int64_t idx = base + k;
    v[k] = idx < n ? in[idx] : 0;
    s += v[k];
  }
  long long tot;
  long long ex = block_exclusive<long long>(s, &tot);
  if (threadIdx.x < 32) {
    // warp-wide look-back: lane l reads the state of tile p - l; a window is
    // used up to its first inclusive prefix once every state up to it is
    // published, otherwise the warp polls again (bounded)
    const int lane = threadIdx.x;
    long long prefix = 0;
    int gave_up = 0;
    if (tile == 0) {
      if (lane == 0) store_state(state, kFlagIncl | ((unsigned long long)tot & kValueMask));
    } else {
      if (lane == 0) store_state(state + tile, kFlagSum | ((unsigned long long)tot & kValueMask));
      long long polls = 0;
      for (int p = tile - 1; p >= 0;) {
        const int q = p - lane;
        // before tile 0 there is an inclusive prefix of zero
        const unsigned long long w = q >= 0 ? load_state(state + q) : kFlagIncl;
        const unsigned long long flag = w & ~kValueMask;
        const unsigned incl = __ballot_sync(0xffffffffu, flag == kFlagIncl);
        const unsigned none = __ballot_sync(0xffffffffu, flag == 0);
        const int first = incl ? __ffs(incl) - 1 : 31;   // last lane of this window to use
        const unsigned used = first == 31 ? 0xffffffffu : ((2u << first) - 1u);
        if (none & used) {
          // an earlier tile has not published yet; its block took its ticket
          // before this one, so it is running
          if (++polls > wait_limit) {
            if (lane == 0) set_error(st, MAFP_ETIMEOUT, tile);
            gave_up = 1;
            break;
          }
          __nanosleep(32);
          continue;
        }
        long long val = lane <= first ? (long long)(w & kValueMask) : 0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) val += __shfl_xor_sync(0xffffffffu, val, o);
        prefix += val;
        if (incl) break;
        p -= 32;
      }
    }
    if (lane == 0) {
      s_prefix = prefix;
      s_gave_up = gave_up;
    }
  }
  __syncthreads();
  if (s_gave_up) {
    // the wait ran out: the whole block sums every value before this tile
    long long acc = 0;
    const int64_t end = (int64_t)tile * kScanTile;
    for (int64_t k = threadIdx.x; k < end; k += kScanThreads) acc += in[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
      long long t = 0;
      for (int w = 0; w < kScanThreads / 32; ++w) t += s_red[w];
      s_prefix = t;
    }
    __syncthreads();
  }
  if (tile > 0 && threadIdx.x == 0)
    store_state(state + tile, kFlagIncl | ((unsigned long long)(s_prefix + tot) & kValueMask));
  ex += s_prefix;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    const int64_t idx = base + k;
    if (idx < n) out[idx] = ex;
    ex += v[k];
  }
  if (tile == ntiles - 1 && threadIdx.x == 0) out[n] = s_prefix + tot;
  // the last block to finish clears the states and tickets for the next scan
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    s_last = atomicAdd(ctr + 1, 1) == ntiles - 1;
  }
  __syncthreads();
  if (s_last) {
    for (int k = threadIdx.x; k < ntiles; k += kScanThreads) store_state(state + k, 0ull);
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
      ctr[0] = 0;
      ctr[1] = 0;
      __threadfence();
    }
  }
}

int scan_i32_to_i64(mafp_ctx *ctx, const int32_t *in, long long *out, int64_t n, cudaStream_t s) {
  if (n <= 0) {
    MAFP_CUDA_TRY(ctx, cudaMemsetAsync(out, 0, sizeof(long long), s));
    return MAFP_OK;
  }
  const int64_t ntiles = (n + kScanTile - 1) / kScanTile;
  const long long limit = ctx->prm.wait_limit > 0 ? (long long)ctx->prm.wait_limit : 0;
  MAFP_TIMED(ctx, s, "k_scan",
             k_scan<<<(unsigned)ntiles, kScanThreads, 0, s>>>(
                 in, out, n, (int)ntiles, reinterpret_cast<unsigned long long *>(ctx->scan_tmp),
                 ctx->scan_ctr, ctx->d_status, limit));
  MAFP_LAUNCH_CHECK(ctx);
  return MAFP_OK;
}

}  // namespace mafp
