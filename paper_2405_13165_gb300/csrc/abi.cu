// abi.cu -- the extern "C" entry points of libmafp.so: argument checks,
// context and scratch management, dispatch to the kernels.
#include <math.h>

#include <algorithm>
#include <stdlib.h>
#include <string.h>

#include "internal.cuh"

namespace mafp {
int build_neighbours(mafp_ctx *, int64_t, int32_t, const void *, int64_t *, int32_t *, int64_t,
                     int64_t *, int32_t *, cudaStream_t);
int build_neighbours_batched(mafp_ctx *, int64_t, int32_t, int32_t, const int64_t *, const void *,
                             int64_t *, int32_t *, int64_t, int64_t *, int32_t *, cudaStream_t);
int cell_order(mafp_ctx *, int64_t, int32_t, const void *, int32_t *, cudaStream_t);
int transpose_map(mafp_ctx *, int64_t, const int64_t *, const int32_t *, uint16_t *,
                  cudaStream_t);
int classify_pca(mafp_ctx *, int64_t, int32_t, const void *, const uint8_t *, const uint8_t *,
                 const void *, const void *, const void *, const uint8_t *, const uint8_t *,
                 const int64_t *, const int32_t *, uint8_t *, uint8_t *, void *, void *, void *,
                 uint8_t *, cudaStream_t);
int build_stencils(mafp_ctx *, int64_t, int32_t, const void *, const uint8_t *, const void *,
                   const int64_t *, const int32_t *, void *, uint8_t *, float *, cudaStream_t);
int build_stencils_backward(mafp_ctx *, int64_t, int32_t, const void *, const uint8_t *,
                            const void *, const int64_t *, const int32_t *, const void *,
                            const void *, void *, cudaStream_t);
int apply_ops(mafp_ctx *, int64_t, int32_t, const int64_t *, const int32_t *, const void *,
              const void *, void *, cudaStream_t);
int apply_ops_backward(mafp_ctx *, int64_t, int32_t, const int64_t *, const int32_t *,
                       const uint16_t *, const void *, const void *, void *, cudaStream_t);
int remap_switched(mafp_ctx *, int64_t, int32_t, const mafp_state *, const uint8_t *,
                   const int64_t *, const int32_t *, const mafp_state *, int64_t, int32_t *,
                   int64_t *, cudaStream_t);
void init_kernel_attributes();
int ghost_sources(mafp_ctx *, int64_t, const uint8_t *, const int64_t *, const int32_t *,
                  uint8_t *, cudaStream_t);
int film_momentum(mafp_ctx *, int64_t, int32_t, const uint8_t *, void *, const void *,
                  const void *, const void *, const void *, const void *, const double *, double,
                  cudaStream_t);
int plane_flux(mafp_ctx *, int64_t, int32_t, const void *, const void *, const void *,
               const void *, const double *, const double *, double *, cudaStream_t);
int normal_stress(mafp_ctx *, int64_t, int32_t, const uint8_t *, const void *, const void *,
                  const void *, double *, cudaStream_t);
int ghost_seed(mafp_ctx *, int64_t, int32_t, const mafp_state *, const uint8_t *,
               const mafp_state *, int64_t, uint8_t *, int32_t *, int64_t *, cudaStream_t);
int ghost_append(mafp_ctx *, int64_t, int64_t, int32_t, const mafp_state *, const mafp_state *,
                 int64_t, int64_t *, cudaStream_t);

int sm_count() {
  static int cached[64] = {0};   // per device; read and written atomically
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) dev = 0;
  int v = __atomic_load_n(&cached[dev], __ATOMIC_ACQUIRE);
  if (!v) {
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    v = v > 0 ? v : 1;
    __atomic_store_n(&cached[dev], v, __ATOMIC_RELEASE);
  }
  return v;
}
}  // namespace mafp

using namespace mafp;
static_assert(kMaxClouds == MAFP_MAX_CLOUDS, "batch limit of the header and the library differ");

static const char *kNoCtx = "null context";

static int fail(mafp_ctx *ctx, int code, const char *msg) {
  if (ctx) snprintf(ctx->err, sizeof(ctx->err), "%s", msg);
  return code;
}

static int check_dtype(mafp_ctx *ctx, int32_t dtype) {
  if (dtype != MAFP_F32_REFINED && dtype != MAFP_F32_PLAIN && dtype != MAFP_F64)
    return fail(ctx, MAFP_EINVAL, "unknown dtype");
  return MAFP_OK;
}

static int check_n(mafp_ctx *ctx, int64_t n) {
  if (n < 0) return fail(ctx, MAFP_EINVAL, "negative particle count");
  if (n > ctx->cap_particles) {
    snprintf(ctx->err, sizeof(ctx->err), "n = %lld exceeds the context capacity %lld",
             (long long)n, (long long)ctx->cap_particles);
    return MAFP_ECAPACITY;
  }
  return MAFP_OK;
}

#define REQUIRE(ptr)                                                   \
  do {                                                                 \
    if (!(ptr)) return fail(ctx, MAFP_EINVAL, "null pointer: " #ptr); \
  } while (0)

static int ensure_device(mafp_ctx *ctx) {
  int cur = -1;
  cudaGetDevice(&cur);
  if (cur != ctx->device) MAFP_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  return MAFP_OK;
}

extern "C" {

void mafp_default_params(mafp_params *p) {
  if (!p) return;
  p->eps_lambda_max = 0.15;
  p->theta_star = M_PI / 6.0;
  p->alpha_film = 4.0;
  p->alpha_w = 4.0;
  p->c_psi = 1.0 / 3.5;
  p->cond_fp64 = 1e4;
  p->eps_band = 1e-4;
  p->angle_band = 1e-3;
  p->hfilm_band = 1e-4;
  p->near_rel = 1e-6;
  p->wait_limit = 4194304.0;
}

int mafp_create(mafp_ctx **out, const mafp_params *params, int64_t cap_particles,
                int64_t cap_cells) {
  if (!out) return MAFP_EINVAL;
  *out = nullptr;
  if (cap_particles < 1 || cap_particles > (int64_t)INT32_MAX - 1) return MAFP_EINVAL;
  if (cap_cells < 1 || cap_cells > (int64_t)INT32_MAX - 1) return MAFP_EINVAL;
  mafp_ctx *ctx = (mafp_ctx *)calloc(1, sizeof(mafp_ctx));
  if (!ctx) return MAFP_ECUDA;
  if (params) ctx->prm = *params; else mafp_default_params(&ctx->prm);
  default_tuning(&ctx->tune);
  ctx->cap_particles = cap_particles;
  ctx->cap_cells = cap_cells;
  cudaGetDevice(&ctx->device);
  int bits = 1;
  while (bits < 32 && ((int64_t)1 << bits) < cap_cells) ++bits;
  ctx->radix_passes = (bits + 7) / 8;
  const int64_t cap = cap_particles;
  ctx->max_tiles = cap / 2048 + 1;
  const int64_t i64_len = std::max<int64_t>(2 * cap + 8, 256 * ctx->max_tiles + 8);
  struct {
    void **p;
    size_t bytes;
  } allocs[] = {
      {(void **)&ctx->keys_a, sizeof(uint32_t) * cap},
      {(void **)&ctx->keys_b, sizeof(uint32_t) * cap},
      {(void **)&ctx->vals_a, sizeof(int32_t) * cap},
      {(void **)&ctx->vals_b, sizeof(int32_t) * cap},
      {(void **)&ctx->radix_hist, sizeof(int32_t) * (256 * ctx->max_tiles + 1)},
      {(void **)&ctx->cell_start, sizeof(int32_t) * cap_cells},
      {(void **)&ctx->cell_end, sizeof(int32_t) * cap_cells},
      {(void **)&ctx->spos, (size_t)(32 * cap)},
      {(void **)&ctx->ucell, sizeof(int32_t) * 2 * cap},
      {(void **)&ctx->n_ucell, sizeof(int32_t) * 8},
      {(void **)&ctx->counts, sizeof(int32_t) * cap},
      {(void **)&ctx->nbr_mask, sizeof(uint32_t) * kMaskWords * cap},
      {(void **)&ctx->overflow, sizeof(int32_t) * cap},
      {(void **)&ctx->scan_tmp, sizeof(long long) * (i64_len / 4096 + 4)},
      {(void **)&ctx->scan_ctr, sizeof(int32_t) * 2},
      {(void **)&ctx->fallback, sizeof(int32_t) * cap},
      {(void **)&ctx->d_status, sizeof(DevStatus)},
      {(void **)&ctx->d_grid, sizeof(GridDev)},
      {(void **)&ctx->d_grids, sizeof(GridDev) * kMaxClouds},
      {(void **)&ctx->cell_base, sizeof(long long) * (kMaxClouds + 1)},
      {(void **)&ctx->cloud_id, sizeof(int32_t) * cap},
      {(void **)&ctx->one_cloud, sizeof(long long) * 2},
      {(void **)&ctx->cloud_partial, sizeof(double) * (kMaxClouds + 16384) * 8},
      {(void **)&ctx->remap_i64, sizeof(int64_t) * i64_len},
      {(void **)&ctx->remap_i32, sizeof(int32_t) * 3 * cap},
  };
  for (auto &a : allocs) {
    cudaError_t e = cudaMalloc(a.p, a.bytes);
    if (e != cudaSuccess) {
      snprintf(ctx->err, sizeof(ctx->err), "cudaMalloc(%zu): %s", a.bytes, cudaGetErrorString(e));
      mafp_destroy(ctx);
      return MAFP_ECUDA;
    }
  }
  if (cudaMemset(ctx->d_status, 0, sizeof(DevStatus)) != cudaSuccess ||
      cudaMemset(ctx->d_grid, 0, sizeof(GridDev)) != cudaSuccess ||
      cudaMemset(ctx->scan_tmp, 0, sizeof(long long) * (i64_len / 4096 + 4)) != cudaSuccess ||
      cudaMemset(ctx->scan_ctr, 0, sizeof(int32_t) * 2) != cudaSuccess) {
    mafp_destroy(ctx);
    return MAFP_ECUDA;
  }
  init_kernel_attributes();
  *out = ctx;
  return MAFP_OK;
}

int mafp_destroy(mafp_ctx *ctx) {
  if (!ctx) return MAFP_OK;
  void *ptrs[] = {ctx->keys_a,    ctx->keys_b,   ctx->vals_a,       ctx->vals_b,
                  ctx->radix_hist, ctx->cell_start, ctx->cell_end,   ctx->spos,
                  ctx->ucell,     ctx->n_ucell,  ctx->counts,       ctx->scan_tmp,
                  ctx->scan_ctr,
                  ctx->nbr_mask,  ctx->overflow,
                  ctx->fallback, ctx->d_status,  ctx->d_grid,
                  ctx->remap_i64, ctx->remap_i32, ctx->d_grids,   ctx->cell_base,
                  ctx->cloud_id,  ctx->one_cloud, ctx->cloud_partial};
  for (void *p : ptrs)
    if (p) cudaFree(p);
  if (ctx->prof_ev) {
    for (int k = 0; k < 2 * kProfCap; ++k) cudaEventDestroy(ctx->prof_ev[k]);
    free(ctx->prof_ev);
    free(ctx->prof_name);
  }
  free(ctx);
  return MAFP_OK;
}

const char *mafp_last_error(const mafp_ctx *ctx) { return ctx ? ctx->err : kNoCtx; }

int mafp_set_tuning(mafp_ctx *ctx, const mafp_tuning *t) {
  if (!ctx || !t) return MAFP_EINVAL;
  const int g3 = t->stencil3d_group, g2 = t->stencil2d_group, ga = t->apply_group;
  const int gb = t->grad3d_group, gf = t->grad2d_group;
  if (!(g3 == 8 || g3 == 16 || g3 == 32)) return fail(ctx, MAFP_EINVAL, "stencil3d_group");
  if (!(g2 == 4 || g2 == 8 || g2 == 16)) return fail(ctx, MAFP_EINVAL, "stencil2d_group");
  if (!(ga == 4 || ga == 8 || ga == 16)) return fail(ctx, MAFP_EINVAL, "apply_group");
  if (!(gb == 2 || gb == 4 || gb == 8 || gb == 16 || gb == 32))
    return fail(ctx, MAFP_EINVAL, "grad3d_group");
  if (!(gf == 1 || gf == 2 || gf == 4 || gf == 8 || gf == 16))
    return fail(ctx, MAFP_EINVAL, "grad2d_group");
  if (t->cell_edge_pct < 100 || t->cell_edge_pct > 200) return fail(ctx, MAFP_EINVAL, "cell_edge_pct");
  const int gc = t->classify_group;
  if (!(gc == 1 || gc == 2 || gc == 4 || gc == 8 || gc == 16))
    return fail(ctx, MAFP_EINVAL, "classify_group");
  ctx->tune = *t;
  return MAFP_OK;
}

int mafp_get_tuning(const mafp_ctx *ctx, mafp_tuning *t) {
  if (!ctx || !t) return MAFP_EINVAL;
  *t = ctx->tune;
  return MAFP_OK;
}

int mafp_get_status(mafp_ctx *ctx, mafp_status *out, void *stream) {
  if (!ctx || !out) return MAFP_EINVAL;
  if (ensure_device(ctx)) return MAFP_ECUDA;
  DevStatus h;
  MAFP_CUDA_TRY(ctx, cudaMemcpyAsync(&h, ctx->d_status, sizeof(h), cudaMemcpyDeviceToHost,
                                     (cudaStream_t)stream));
  MAFP_CUDA_TRY(ctx, cudaStreamSynchronize((cudaStream_t)stream));
  out->code = h.code;
  out->cells_identity = h.cells_identity;
  out->required = h.required;
  out->nnz = h.nnz;
  out->n_fp64_stencil = h.n_fp64_stencil;
  out->n_fp64_eigen = h.n_fp64_eigen;
  out->n_deficient = h.n_deficient;
  out->n_near = h.n_near;
  out->n_out = h.n_out;
  out->n_nonfinite = h.n_nonfinite;
  out->ncells = h.ncells;
  out->cell_size = h.cell_size;
  return MAFP_OK;
}

int mafp_reset_status(mafp_ctx *ctx, void *stream) {
  if (!ctx) return MAFP_EINVAL;
  if (ensure_device(ctx)) return MAFP_ECUDA;
  MAFP_CUDA_TRY(ctx, cudaMemsetAsync(ctx->d_status, 0, sizeof(DevStatus), (cudaStream_t)stream));
  return MAFP_OK;
}

int mafp_build_neighbours(mafp_ctx *ctx, int64_t n, int32_t dtype, const void *pos_h,
                          int64_t *row_ptr, int32_t *col, int64_t cap_nnz, int64_t *nnz_dev,
                          int32_t *order, void *stream) {
  if (!ctx) return MAFP_EINVAL;
  int rc;
  if ((rc = check_dtype(ctx, dtype)) || (rc = check_n(ctx, n))) return rc;
  REQUIRE(row_ptr);
  if (cap_nnz < 0) return fail(ctx, MAFP_EINVAL, "negative cap_nnz");
  if (ensure_device(ctx)) return MAFP_ECUDA;
  cudaStream_t s = (cudaStream_t)stream;
  if (n == 0) {
    MAFP_CUDA_TRY(ctx, cudaMemsetAsync(row_ptr, 0, sizeof(int64_t), s));
    if (nnz_dev) MAFP_CUDA_TRY(ctx, cudaMemsetAsync(nnz_dev, 0, sizeof(int64_t), s));
    return MAFP_OK;
  }
  REQUIRE(pos_h);
  REQUIRE(col);
  return build_neighbours(ctx, n, dtype, pos_h, row_ptr, col, cap_nnz, nnz_dev, order, s);
}

int mafp_cell_order(mafp_ctx *ctx, int64_t n, int32_t dtype, const void *pos_h, int32_t *order,
                    void *stream) {
  if (!ctx) return MAFP_EINVAL;
  int rc;
  if ((rc = check_dtype(ctx, dtype)) || (rc = check_n(ctx, n))) return rc;
  if (n == 0) return MAFP_OK;
  REQUIRE(pos_h);
  REQUIRE(order);
  if (ensure_device(ctx)) return MAFP_ECUDA;
  return cell_order(ctx, n, dtype, pos_h, order, (cudaStream_t)stream);
}

int mafp_build_neighbours_batched(mafp_ctx *ctx, int64_t n, int32_t dtype, int32_t nclouds,
                                  const int64_t *cloud_offset, const void *pos_h,
                                  int64_t *row_ptr, int32_t *col, int64_t cap_nnz,
                                  int64_t *nnz_dev, int32_t *order, void *stream) {
  if (!ctx) return MAFP_EINVAL;
  int rc;
  if ((rc = check_dtype(ctx, dtype)) || (rc = check_n(ctx, n))) return rc;
  if (nclouds < 1 || nclouds > kMaxClouds) return fail(ctx, MAFP_EINVAL, "nclouds out of range");
  REQUIRE(row_ptr);
  REQUIRE(cloud_offset);
  if (cap_nnz < 0) return fail(ctx, MAFP_EINVAL, "negative cap_nnz");
  if (ensure_device(ctx)) return MAFP_ECUDA;
  cudaStream_t s = (cudaStream_t)stream;
  if (n == 0) {
    MAFP_CUDA_TRY(ctx, cudaMemsetAsync(row_ptr, 0, sizeof(int64_t), s));
    if (nnz_dev) MAFP_CUDA_TRY(ctx, cudaMemsetAsync(nnz_dev, 0, sizeof(int64_t), s));
    return MAFP_OK;
  }
  REQUIRE(pos_h);
  REQUIRE(col);
  return build_neighbours_batched(ctx, n, dtype, nclouds, cloud_offset, pos_h, row_ptr, col,
                                  cap_nnz, nnz_dev, order, s);
}

int mafp_classify_pca(mafp_ctx *ctx, int64_t n, int32_t dtype, const void *pos_h,
                      const uint8_t *model, const uint8_t *type, const void *normal,
                      const void *vol, const void *h3d, const uint8_t *user,
                      const uint8_t *last, const int64_t *row_ptr, const int32_t *col,
                      uint8_t *flag, uint8_t *preflag, void *eig, void *frame, void *hfilm,
                      uint8_t *near, void *stream) {
  if (!ctx) return MAFP_EINVAL;
  int rc;
  if ((rc = check_dtype(ctx, dtype)) || (rc = check_n(ctx, n))) return rc;
  if (n == 0) return MAFP_OK;
  REQUIRE(pos_h); REQUIRE(model); REQUIRE(type); REQUIRE(normal); REQUIRE(vol); REQUIRE(h3d);
  REQUIRE(user); REQUIRE(last); REQUIRE(row_ptr); REQUIRE(col); REQUIRE(flag); REQUIRE(preflag);
  REQUIRE(eig); REQUIRE(frame); REQUIRE(hfilm);
  if (ensure_device(ctx)) return MAFP_ECUDA;
  return classify_pca(ctx, n, dtype, pos_h, model, type, normal, vol, h3d, user, last, row_ptr,
                      col, flag, preflag, eig, frame, hfilm, near, (cudaStream_t)stream);
}

int mafp_build_stencils(mafp_ctx *ctx, int64_t n, int32_t dtype, const void *pos_h,
                        const uint8_t *model, const void *frame, const int64_t *row_ptr,
                        const int32_t *col, void *coef, uint8_t *status, float *cond,
                        void *stream) {
  if (!ctx) return MAFP_EINVAL;
  int rc;
  if ((rc = check_dtype(ctx, dtype)) || (rc = check_n(ctx, n))) return rc;
  if (n == 0) return MAFP_OK;
  REQUIRE(pos_h); REQUIRE(model); REQUIRE(frame); REQUIRE(row_ptr); REQUIRE(col); REQUIRE(coef);
  REQUIRE(status); REQUIRE(cond);
  if (ensure_device(ctx)) return MAFP_ECUDA;
  return build_stencils(ctx, n, dtype, pos_h, model, frame, row_ptr, col, coef, status, cond,
                        (cudaStream_t)stream);
}

int mafp_apply_ops(mafp_ctx *ctx, int64_t n, int32_t dtype, const int64_t *row_ptr,
                   const int32_t *col, const void *coef, const void *fields, void *out,
                   void *stream) {
  if (!ctx) return MAFP_EINVAL;
  int rc;
  if ((rc = check_dtype(ctx, dtype))) return rc;
  if (n < 0) return fail(ctx, MAFP_EINVAL, "negative particle count");
  if (n == 0) return MAFP_OK;
  REQUIRE(row_ptr); REQUIRE(col); REQUIRE(coef); REQUIRE(fields); REQUIRE(out);
  if (ensure_device(ctx)) return MAFP_ECUDA;
  return apply_ops(ctx, n, dtype, row_ptr, col, coef, fields, out, (cudaStream_t)stream);
}

int mafp_transpose_map(mafp_ctx *ctx, int64_t n, const int64_t *row_ptr, const int32_t *col,
                       uint16_t *tloc, void *stream) {
  if (!ctx) return MAFP_EINVAL;
  if (n < 0) return fail(ctx, MAFP_EINVAL, "negative particle count");
  if (n == 0) return MAFP_OK;
  REQUIRE(row_ptr); REQUIRE(col); REQUIRE(tloc);
  if (ensure_device(ctx)) return MAFP_ECUDA;
  return transpose_map(ctx, n, row_ptr, col, tloc, (cudaStream_t)stream);
}

int mafp_apply_ops_backward(mafp_ctx *ctx, int64_t n, int32_t dtype, const int64_t *row_ptr,
                            const int32_t *col, const uint16_t *tloc, const void *coef,
                            const void *gout, void *gfields, void *stream) {
  if (!ctx) return MAFP_EINVAL;
  int rc;
  if ((rc = check_dtype(ctx, dtype))) return rc;
  if (n < 0) return fail(ctx, MAFP_EINVAL, "negative particle count");
  if (n == 0) return MAFP_OK;
  REQUIRE(row_ptr); REQUIRE(col); REQUIRE(coef); REQUIRE(gout); REQUIRE(gfields);
  if (ensure_device(ctx)) return MAFP_ECUDA;
  return apply_ops_backward(ctx, n, dtype, row_ptr, col, tloc, coef, gout, gfields,
                            (cudaStream_t)stream);
}

int mafp_build_stencils_backward(mafp_ctx *ctx, int64_t n, int32_t dtype, const void *pos_h,
                                 const uint8_t *model, const void *frame,
                                 const int64_t *row_ptr, const int32_t *col,
                                 const void *fields, const void *gout, void *gpos,
                                 void *stream) {
  if (!ctx) return MAFP_EINVAL;
  int rc;
  if ((rc = check_dtype(ctx, dtype)) || (rc = check_n(ctx, n))) return rc;
  if (n == 0) return MAFP_OK;
  REQUIRE(pos_h); REQUIRE(model); REQUIRE(frame); REQUIRE(row_ptr); REQUIRE(col);
  REQUIRE(fields); REQUIRE(gout); REQUIRE(gpos);
  if (ensure_device(ctx)) return MAFP_ECUDA;
  return build_stencils_backward(ctx, n, dtype, pos_h, model, frame, row_ptr, col, fields, gout,
                                 gpos, (cudaStream_t)stream);
}

int mafp_film_momentum(mafp_ctx *ctx, int64_t n, int32_t dtype, const uint8_t *model, void *vp,
                       const void *rho, const void *eta, const void *hfilm, const void *normal,
                       const void *out, const double *gravity, double dt, void *stream) {
  if (!ctx) return MAFP_EINVAL;
  int rc;
  if ((rc = check_dtype(ctx, dtype))) return rc;
  if (n < 0) return fail(ctx, MAFP_EINVAL, "negative particle count");
  if (n == 0) return MAFP_OK;
  REQUIRE(model); REQUIRE(vp); REQUIRE(rho); REQUIRE(eta); REQUIRE(hfilm); REQUIRE(normal);
  REQUIRE(out); REQUIRE(gravity);
  if (!(dt >= 0.0)) return fail(ctx, MAFP_EINVAL, "dt must be >= 0");
  if (ensure_device(ctx)) return MAFP_ECUDA;
  return film_momentum(ctx, n, dtype, model, vp, rho, eta, hfilm, normal, out, gravity, dt,
                       (cudaStream_t)stream);
}

int mafp_plane_flux(mafp_ctx *ctx, int64_t n, int32_t dtype, const void *pos_old,
                    const void *pos_new, const void *mass, const void *rho, const double *point,
                    const double *normal, double *acc_dev, void *stream) {
  if (!ctx) return MAFP_EINVAL;
  int rc;
  if ((rc = check_dtype(ctx, dtype))) return rc;
  if (n < 0) return fail(ctx, MAFP_EINVAL, "negative particle count");
  if (n == 0) return MAFP_OK;
  REQUIRE(pos_old); REQUIRE(pos_new); REQUIRE(mass); REQUIRE(rho); REQUIRE(point);
  REQUIRE(normal); REQUIRE(acc_dev);
  if (ensure_device(ctx)) return MAFP_ECUDA;
  return plane_flux(ctx, n, dtype, pos_old, pos_new, mass, rho, point, normal, acc_dev,
                    (cudaStream_t)stream);
}

int mafp_normal_stress(mafp_ctx *ctx, int64_t n, int32_t dtype, const uint8_t *select,
                       const void *out, const void *eta, const void *normal, double *acc_dev,
                       void *stream) {
  if (!ctx) return MAFP_EINVAL;
  int rc;
  if ((rc = check_dtype(ctx, dtype))) return rc;
  if (n < 0) return fail(ctx, MAFP_EINVAL, "negative particle count");
  if (n == 0) return MAFP_OK;
  REQUIRE(select); REQUIRE(out); REQUIRE(eta); REQUIRE(normal); REQUIRE(acc_dev);
  if (ensure_device(ctx)) return MAFP_ECUDA;
  return normal_stress(ctx, n, dtype, select, out, eta, normal, acc_dev, (cudaStream_t)stream);
}

int mafp_ghost_sources(mafp_ctx *ctx, int64_t n, const uint8_t *model, const int64_t *row_ptr,
                       const int32_t *col, uint8_t *src, void *stream) {
  if (!ctx) return MAFP_EINVAL;
  int rc;
  if ((rc = check_n(ctx, n))) return rc;
  if (n == 0) return MAFP_OK;
  REQUIRE(model); REQUIRE(row_ptr); REQUIRE(col); REQUIRE(src);
  if (ensure_device(ctx)) return MAFP_ECUDA;
  return ghost_sources(ctx, n, model, row_ptr, col, src, (cudaStream_t)stream);
}

int mafp_ghost_seed(mafp_ctx *ctx, int64_t n, int32_t dtype, const mafp_state *in,
                    const uint8_t *src, const mafp_state *ghost, int64_t cap_ghost,
                    uint8_t *ghost_flag, int32_t *ghost_src, int64_t *n_ghost_dev,
                    void *stream) {
  if (!ctx) return MAFP_EINVAL;
  int rc;
  if ((rc = check_dtype(ctx, dtype)) || (rc = check_n(ctx, n))) return rc;
  if (cap_ghost < 0) return fail(ctx, MAFP_EINVAL, "negative cap_ghost");
  REQUIRE(in); REQUIRE(src); REQUIRE(ghost); REQUIRE(ghost_flag); REQUIRE(ghost_src);
  if (ensure_device(ctx)) return MAFP_ECUDA;
  if (n == 0) {
    if (n_ghost_dev)
      MAFP_CUDA_TRY(ctx, cudaMemsetAsync(n_ghost_dev, 0, sizeof(int64_t), (cudaStream_t)stream));
    return MAFP_OK;
  }
  return ghost_seed(ctx, n, dtype, in, src, ghost, cap_ghost, ghost_flag, ghost_src,
                    n_ghost_dev, (cudaStream_t)stream);
}

int mafp_ghost_append(mafp_ctx *ctx, int64_t n_regular, int64_t n_ghost, int32_t dtype,
                      const mafp_state *ghost, const mafp_state *all, int64_t cap_all,
                      int64_t *n_all_dev, void *stream) {
  if (!ctx) return MAFP_EINVAL;
  int rc;
  if ((rc = check_dtype(ctx, dtype)) || (rc = check_n(ctx, n_ghost))) return rc;
  if (n_regular < 0 || cap_all < n_regular)
    return fail(ctx, MAFP_EINVAL, "n_regular must lie in [0, cap_all]");
  REQUIRE(ghost); REQUIRE(all);
  if (ensure_device(ctx)) return MAFP_ECUDA;
  return ghost_append(ctx, n_regular, n_ghost, dtype, ghost, all, cap_all, n_all_dev,
                      (cudaStream_t)stream);
}

int mafp_remap_switched(mafp_ctx *ctx, int64_t n, int32_t dtype, const mafp_state *in,
                        const uint8_t *flag, const int64_t *row_ptr, const int32_t *col,
                        const mafp_state *out, int64_t cap_out, int32_t *old2new,
                        int64_t *n_out_dev, void *stream) {
  if (!ctx) return MAFP_EINVAL;
  int rc;
  if ((rc = check_dtype(ctx, dtype)) || (rc = check_n(ctx, n))) return rc;
  REQUIRE(in); REQUIRE(out); REQUIRE(flag); REQUIRE(row_ptr); REQUIRE(col); REQUIRE(old2new);
  if (cap_out < 0) return fail(ctx, MAFP_EINVAL, "negative cap_out");
  if (ensure_device(ctx)) return MAFP_ECUDA;
  if (n == 0) {
    if (n_out_dev) MAFP_CUDA_TRY(ctx, cudaMemsetAsync(n_out_dev, 0, sizeof(int64_t),
                                                      (cudaStream_t)stream));
    return MAFP_OK;
  }
  const void *ptrs[] = {in->pos_h, in->vp, in->normal, in->rho, in->eta, in->mass, in->diam,
                        in->hfilm, in->h3d, in->model, in->type, in->last,
                        out->pos_h, out->vp, out->normal, out->rho, out->eta, out->mass,
                        out->diam, out->hfilm, out->h3d, out->model, out->type, out->last};
  for (const void *p : ptrs)
    if (!p) return fail(ctx, MAFP_EINVAL, "null array in mafp_state");
  return remap_switched(ctx, n, dtype, in, flag, row_ptr, col, out, cap_out, old2new, n_out_dev,
                        (cudaStream_t)stream);
}

int mafp_profile(mafp_ctx *ctx, int32_t enable) {
  if (!ctx) return MAFP_EINVAL;
  if (ensure_device(ctx)) return MAFP_ECUDA;
  if (enable && !ctx->prof_ev) {
    ctx->prof_ev = (cudaEvent_t *)calloc(2 * kProfCap, sizeof(cudaEvent_t));
    ctx->prof_name = (const char **)calloc(kProfCap, sizeof(const char *));
    if (!ctx->prof_ev || !ctx->prof_name) return fail(ctx, MAFP_ECUDA, "out of host memory");
    for (int k = 0; k < 2 * kProfCap; ++k) MAFP_CUDA_TRY(ctx, cudaEventCreate(&ctx->prof_ev[k]));
  }
  if (enable) ctx->prof_n = 0;
  ctx->prof_on = enable ? 1 : 0;
  return MAFP_OK;
}

int mafp_profile_read(mafp_ctx *ctx, mafp_kernel_time *out, int32_t cap, int32_t *count) {
  if (!ctx || !count || (cap > 0 && !out)) return MAFP_EINVAL;
  if (ensure_device(ctx)) return MAFP_ECUDA;
  *count = 0;
  if (!ctx->prof_ev) return MAFP_OK;
  MAFP_CUDA_TRY(ctx, cudaDeviceSynchronize());
  int m = 0;
  for (int k = 0; k < ctx->prof_n; ++k) {
    float ms = 0.0f;
    MAFP_CUDA_TRY(ctx, cudaEventElapsedTime(&ms, ctx->prof_ev[2 * k], ctx->prof_ev[2 * k + 1]));
    int slot = -1;
    for (int q = 0; q < m; ++q)
      if (strncmp(out[q].name, ctx->prof_name[k], sizeof(out[q].name) - 1) == 0) slot = q;
    if (slot < 0) {
      if (m >= cap) continue;
      slot = m++;
      memset(&out[slot], 0, sizeof(out[slot]));
      strncpy(out[slot].name, ctx->prof_name[k], sizeof(out[slot].name) - 1);
    }
    out[slot].launches += 1;
    out[slot].total_ms += ms;
  }
  *count = m;
  return MAFP_OK;
}

}  // extern "C"
