// ghost.cu -- the buffer zone of Sec. 5.3 (Alg. 5).
//  sources:  particle i is a source when S_i holds a particle of the other model;
//  seed:     every source is copied, in index order, as an intermediate ghost,
//            with the transition it takes (3D wall -> 2D, 2D -> 3D; interior /
//            free-surface 3D ghosts are the candidates Alg. 3 maps onto walls);
//  append:   after the transition (mafp_remap_switched on the ghost cloud), the
//            ghosts it produced are appended behind the regular particles.
#include "internal.cuh"
#include "state.cuh"

namespace mafp {

__global__ void k_ghost_sources(int64_t n, const uint8_t *model, const long long *row_ptr,
                                const int32_t *col, uint8_t *src) {
  const int lane = threadIdx.x & 31;
  const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i = wid; i < n; i += nwarps) {
    const uint8_t mi = model[i];
    int other = 0;
    for (long long e = row_ptr[i] + lane; e < row_ptr[i + 1]; e += 32)
      other |= model[col[e]] != mi ? 1 : 0;
    other = __any_sync(0xffffffffu, other);
    if (lane == 0) src[i] = (uint8_t)other;
  }
}

__global__ void k_u8_to_i32(int64_t n, const uint8_t *a, uint8_t want, int32_t *out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = a[i] == want ? 1 : 0;
}

// Total of a selection (exclusive scan `off`, n entries) placed after `base`
// rows: writes the count, flags a capacity overflow (nothing is then copied).
__global__ void k_select_total(const long long *off, int64_t n, int64_t base, long long cap,
                               int64_t *n_dev, DevStatus *st) {
  const long long total = base + off[n];
  if (n_dev) *n_dev = total;
  st->remap_scratch[1] = total > cap ? 1 : 0;
  if (total > cap) set_error(st, MAFP_ECAPACITY, total);
}

template <typename T>
__global__ void k_ghost_seed(int64_t n, StateT<T> in, const uint8_t *src, const long long *off,
                             StateT<T> g, uint8_t *gflag, int32_t *gsrc, const DevStatus *st) {
  if (st->remap_scratch[1] != 0) return;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    if (!src[i]) continue;
    const long long o = off[i];
    copy_particle(in, i, g, o);
    g.last[o] = 0;
    const uint8_t m = in.model[i];
    gflag[o] = m == MAFP_MODEL_2D ? 2 : (in.type[i] == MAFP_TYPE_WALL ? 1 : 0);
    gsrc[o] = (int32_t)i;
  }
}

template <typename T>
__global__ void k_ghost_append(int64_t ng, StateT<T> gf, const long long *off, StateT<T> all,
                               int64_t base, const DevStatus *st) {
  if (st->remap_scratch[1] != 0) return;
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < ng;
       g += (int64_t)gridDim.x * blockDim.x) {
    if (gf.last[g] != 1) continue;
    copy_particle(gf, g, all, base + off[g]);
  }
}

int ghost_sources(mafp_ctx *ctx, int64_t n, const uint8_t *model, const int64_t *row_ptr,
                  const int32_t *col, uint8_t *src, cudaStream_t s) {
  const int sms = sm_count();
  MAFP_TIMED(ctx, s, "k_ghost_sources",
             k_ghost_sources<<<grid_for(n * 32, 256, sms * 32), 256, 0, s>>>(
                 n, model, reinterpret_cast<const long long *>(row_ptr), col, src));
  MAFP_LAUNCH_CHECK(ctx);
  return MAFP_OK;
}

template <typename T>
static int ghost_seed_t(mafp_ctx *ctx, int64_t n, const mafp_state *in_, const uint8_t *src,
                        const mafp_state *g_, int64_t cap_ghost, uint8_t *gflag, int32_t *gsrc,
                        int64_t *n_ghost_dev, cudaStream_t s) {
  const StateT<T> in = cast_state<T>(in_), g = cast_state<T>(g_);
  long long *off = reinterpret_cast<long long *>(ctx->remap_i64);
  const int sms = sm_count();
  MAFP_TIMED(ctx, s, "k_u8_to_i32",
             k_u8_to_i32<<<grid_for(n, 256, sms * 16), 256, 0, s>>>(n, src, 1, ctx->counts));
  int rc = scan_i32_to_i64(ctx, ctx->counts, off, n, s);
  if (rc) return rc;
  MAFP_TIMED(ctx, s, "k_select_total",
             k_select_total<<<1, 1, 0, s>>>(off, n, 0, cap_ghost, n_ghost_dev, ctx->d_status));
  MAFP_TIMED(ctx, s, "k_ghost_seed<T>",
             k_ghost_seed<T><<<grid_for(n, 256, sms * 16), 256, 0, s>>>(n, in, src, off, g, gflag,
                                                                      gsrc, ctx->d_status));
  MAFP_LAUNCH_CHECK(ctx);
  return MAFP_OK;
}

template <typename T>
static int ghost_append_t(mafp_ctx *ctx, int64_t n_regular, int64_t n_ghost,
                          const mafp_state *gf_, const mafp_state *all_, int64_t cap_all,
                          int64_t *n_all_dev, cudaStream_t s) {
  const StateT<T> gf = cast_state<T>(gf_), all = cast_state<T>(all_);
  long long *off = reinterpret_cast<long long *>(ctx->remap_i64);
  const int sms = sm_count();
  MAFP_TIMED(ctx, s, "k_u8_to_i32",
             k_u8_to_i32<<<grid_for(n_ghost, 256, sms * 16), 256, 0, s>>>(n_ghost, gf.last, 1,
                                                                         ctx->counts));
  int rc = scan_i32_to_i64(ctx, ctx->counts, off, n_ghost, s);
  if (rc) return rc;
  MAFP_TIMED(ctx, s, "k_select_total",
             k_select_total<<<1, 1, 0, s>>>(off, n_ghost, n_regular, cap_all, n_all_dev,
                                            ctx->d_status));
  MAFP_TIMED(ctx, s, "k_ghost_append<T>",
             k_ghost_append<T><<<grid_for(n_ghost, 256, sms * 16), 256, 0, s>>>(
                 n_ghost, gf, off, all, n_regular, ctx->d_status));
  MAFP_LAUNCH_CHECK(ctx);
  return MAFP_OK;
}

int ghost_seed(mafp_ctx *ctx, int64_t n, int32_t dtype, const mafp_state *in, const uint8_t *src,
               const mafp_state *g, int64_t cap_ghost, uint8_t *gflag, int32_t *gsrc,
               int64_t *n_ghost_dev, cudaStream_t s) {
  if (dtype == MAFP_F64)
    return ghost_seed_t<double>(ctx, n, in, src, g, cap_ghost, gflag, gsrc, n_ghost_dev, s);
  return ghost_seed_t<float>(ctx, n, in, src, g, cap_ghost, gflag, gsrc, n_ghost_dev, s);
}

int ghost_append(mafp_ctx *ctx, int64_t n_regular, int64_t n_ghost, int32_t dtype,
                 const mafp_state *gf, const mafp_state *all, int64_t cap_all, int64_t *n_all_dev,
                 cudaStream_t s) {
  if (dtype == MAFP_F64)
    return ghost_append_t<double>(ctx, n_regular, n_ghost, gf, all, cap_all, n_all_dev, s);
  return ghost_append_t<float>(ctx, n_regular, n_ghost, gf, all, cap_all, n_all_dev, s);
}

}  // namespace mafp
