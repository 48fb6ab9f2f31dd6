/* mafp.h -- C ABI of libmafp.so: the per-particle operator pipeline of the
 * meshfree 3D/2D model-adaptive flow method (Suchde, "Adaptive coupling of 3D
 * and 2D fluid flow models", arXiv 2405.13165) on one GB300 (sm_103a).
 *
 * General rules for every entry point
 *  - Pointers named *_dev / arrays of particles are DEVICE pointers owned by
 *    the caller; the library never frees or keeps them after the call returns.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Calls only enqueue work and return; results are ready once the
 *    stream reaches the enqueued work.  Nothing allocates after mafp_create.
 *  - Return value: MAFP_OK (0) or a negative MAFP_E* code for errors found on
 *    the host (bad arguments, capacity known to be too small, CUDA launch
 *    failure).  Conditions only the device can see (a nnz larger than the
 *    col capacity, non-finite input, a remap needing more output rows) are
 *    recorded in the context's device status block: read it with
 *    mafp_get_status after the stream is done.
 *  - Calls of one context must be ordered on the GPU (one stream, or streams
 *    ordered by events): they share the context's scratch, so calls that
 *    overlap on the GPU race on it.  Different contexts are independent.
 *  - Particle arrays are in the caller's order; all indices refer to it.
 *  - dtype selects the floating-point type of every "void*" real array of
 *    the call: float for MAFP_F32_REFINED / MAFP_F32_PLAIN, double for
 *    MAFP_F64.  "x4" arrays hold 4 reals per particle (16 or 32 bytes).
 */
#ifndef MAFP_H
#define MAFP_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define MAFP_OK 0
#define MAFP_EINVAL (-1)     /* bad argument (null pointer, negative size, unknown dtype) */
#define MAFP_ECAPACITY (-2)  /* a caller or context capacity is too small */
#define MAFP_ECUDA (-3)      /* a CUDA runtime call failed (message in mafp_last_error) */
#define MAFP_ETIMEOUT (-4)   /* a bounded device-side wait gave up (status block); the
                                waiting block then computed the value itself, so the
                                outputs are exact but the call ran its slow path */
#define MAFP_ENOTIMPL (-5)   /* entry point not implemented by this library */
#define MAFP_ENONFINITE (-6) /* non-finite position or smoothing length seen on device */

/* precision of a call */
#define MAFP_F32_REFINED 0   /* FP32 with one refinement step, FP64 retakes where needed */
#define MAFP_F32_PLAIN 1     /* FP32, no refinement */
#define MAFP_F64 2           /* FP64 throughout */

/* particle model / type codes (Sec. 2.3, Sec. 4.2) */
#define MAFP_MODEL_3D 0
#define MAFP_MODEL_2D 1
#define MAFP_TYPE_INTERIOR 0
#define MAFP_TYPE_FREE_SURFACE 1
#define MAFP_TYPE_WALL 2
/* user-defined criterion bits (Alg. 2, Sec. 4.2) */
#define MAFP_USER_TO_2D 1
#define MAFP_USER_TO_3D 2
/* per-particle stencil status */
#define MAFP_STENCIL_OK 0
#define MAFP_STENCIL_DEFICIENT 1  /* moment matrix rank deficient: coefficients zero */
#define MAFP_STENCIL_FP64 2       /* OK, recomputed in FP64 (condition estimate too large) */

typedef struct mafp_ctx mafp_ctx;

typedef struct {
  double eps_lambda_max; /* Eq. EigenvalueLimit threshold (paper: 0.15) */
  double theta_star;     /* Eq. EigenvectorLimit max deviation (paper: pi/6) */
  double alpha_film;     /* alpha of Eq. Height (not given in the paper; default 4) */
  double alpha_w;        /* shape of the GFDM weight W(s) (not given; default 4) */
  double c_psi;          /* (r_min + r_max)/2 of Sec. 5.2 (not given; default 1/3.5) */
  double cond_fp64;      /* FP32 stencils whose condition estimate exceeds this are redone in FP64 (1e4) */
  double eps_band;       /* FP32 eps_lambda within this of its threshold -> FP64 retake */
  double angle_band;     /* FP32 |n.w3| within this of cos(theta*) -> FP64 retake */
  double hfilm_band;     /* FP32 H_film within this relative band of h3D -> FP64 retake */
  double near_rel;       /* relative band for reporting near-threshold decisions (1e-6) */
  double wait_limit;     /* polls of a bounded device-side wait (the one-pass scan's wait
                            for an earlier tile) before it gives up and records
                            MAFP_ETIMEOUT in the status block (2^22); no counterpart in
                            the paper */
} mafp_params;

/* Launch shapes (no counterpart in the paper): lanes that cooperate on one
 * particle or row.  Every value gives the same results up to rounding order;
 * the autotuner picks the fastest for a cloud's population mix. */
typedef struct {
  int32_t stencil3d_group; /* lanes per 3D particle in mafp_build_stencils: 8, 16 or 32 */
  int32_t stencil2d_group; /* lanes per 2D particle in mafp_build_stencils: 4, 8 or 16 */
  int32_t apply_group;     /* lanes per row in mafp_apply_ops / _backward: 4, 8 or 16 */
  int32_t grad3d_group;    /* lanes per 3D particle in mafp_build_stencils_backward: 2, 4,
                              8, 16 or 32 (the FP64 adjoint takes at least 8) */
  int32_t grad2d_group;    /* lanes per 2D particle in mafp_build_stencils_backward: 1, 2,
                              4, 8 or 16 */
  int32_t cell_edge_pct;   /* cell tile of the neighbour search: the grid's cell edge in
                              percent of the cloud's largest h, 100..200 (larger cells:
                              more candidates per particle, fewer cells to stage); the
                              neighbour sets are the same for every value */
  int32_t classify_group;  /* lanes per particle in mafp_classify_pca: 1, 2, 4, 8 or 16 */
} mafp_tuning;

/* Device-side status block, copied out by mafp_get_status. */
typedef struct {
  int32_t code;            /* first device-detected error (MAFP_E*), 0 if none */
  int32_t cells_identity;  /* 1 if the last cell sort left the particle order unchanged */
  int64_t required;        /* capacity that would have been needed (code == MAFP_ECAPACITY) */
  int64_t nnz;             /* nnz of the last mafp_build_neighbours */
  int64_t n_fp64_stencil;  /* particles whose stencil was redone in FP64 */
  int64_t n_fp64_eigen;    /* detection decisions retaken in FP64 */
  int64_t n_deficient;     /* rank-deficient stencils */
  int64_t n_near;          /* detection decisions within near_rel of their threshold */
  int64_t n_out;           /* particle count produced by the last remap */
  int64_t n_nonfinite;     /* non-finite positions / smoothing lengths seen */
  int64_t ncells;          /* cells of the last neighbour grid */
  double cell_size;        /* edge of the last neighbour grid's cells */
} mafp_status;

/* Fill *p with the defaults listed above. */
void mafp_default_params(mafp_params *p);

/* Create a context for clouds of up to cap_particles particles whose
 * neighbour grid has up to cap_cells cells (the cell edge grows beyond max h
 * when the bounding box would need more).  Allocates all device scratch
 * (about 60 bytes per particle + 8 bytes per cell) on the current device.
 * params may be NULL (defaults).  Returns MAFP_OK and *out, or MAFP_EINVAL /
 * MAFP_ECUDA. */
int mafp_create(mafp_ctx **out, const mafp_params *params, int64_t cap_particles,
                int64_t cap_cells);
/* Free the context and its scratch.  NULL is accepted. */
int mafp_destroy(mafp_ctx *ctx);
/* Message of the last host-side error of this context (never NULL). */
const char *mafp_last_error(const mafp_ctx *ctx);
/* Set / read the launch shapes of a context (MAFP_EINVAL for unsupported values). */
int mafp_set_tuning(mafp_ctx *ctx, const mafp_tuning *t);
int mafp_get_tuning(const mafp_ctx *ctx, mafp_tuning *t);
/* Copy the device status block to *out after synchronising `stream`. */
int mafp_get_status(mafp_ctx *ctx, mafp_status *out, void *stream);
/* Zero the device status block (enqueued on `stream`). */
int mafp_reset_status(mafp_ctx *ctx, void *stream);

/* --------------------------------------------------------------------------
 * mafp_build_neighbours -- neighbourhoods S_i of Eq. Nbd (Sec. 2.2):
 *   S_i = { j : |x_j - x_i| <= (h_i + h_j)/2 },  i in S_i,
 * over all n particles of both models, evaluated as
 *   d^2 = (dx*dx + dy*dy) + dz*dz <= ((h_i + h_j) * 0.5)^2,  dx = x_j - x_i,
 * the FP32 path retaking every pair within a 1e-5 relative band in FP64 so
 * the sets are those of the FP64 definition.  Built on a cell list: cell keys
 * of edge >= max h, a stable LSD radix sort of (key, index), 27-cell search.
 *   pos_h    x4 [n]        x, y, z, h (h = support radius)
 *   row_ptr  int64 [n+1]   written: CSR row starts, row_ptr[n] = nnz
 *   col      int32 [cap_nnz] written: column indices, each row ascending
 *   nnz_dev  int64 [1]     written: nnz (also in the status block)
 *   order    int32 [n] or NULL: written: cell order (sorted position -> index);
 *            reordering a cloud by it makes later calls take the fast path
 * If nnz > cap_nnz, row_ptr is still written, col is not, and the status
 * block records MAFP_ECAPACITY with required = nnz. */
int mafp_build_neighbours(mafp_ctx *ctx, int64_t n, int32_t dtype, const void *pos_h,
                          int64_t *row_ptr, int32_t *col, int64_t cap_nnz, int64_t *nnz_dev,
                          int32_t *order, void *stream);

/* mafp_cell_order -- the first stage of mafp_build_neighbours alone (grid of
 * edge >= max h over the bounding box, cell keys, stable radix sort): writes
 * the permutation that puts the particles in cell order, order[s] = index of
 * the particle at sorted position s, without building neighbour lists.  A
 * time loop re-sorts its particles by it so the next neighbour build takes
 * the in-order path.  order int32 [n] written; the status block reports
 * cells_identity as mafp_build_neighbours does. */
int mafp_cell_order(mafp_ctx *ctx, int64_t n, int32_t dtype, const void *pos_h, int32_t *order,
                    void *stream);

/* Largest nclouds of mafp_build_neighbours_batched. */
#define MAFP_MAX_CLOUDS 65536

/* --------------------------------------------------------------------------
 * mafp_build_neighbours_batched -- Eq. Nbd for nclouds independent clouds
 * stored back to back: cloud b owns particles [cloud_offset[b],
 * cloud_offset[b+1]), and S_i only ever holds particles of i's own cloud
 * (each cloud gets its own bounding box and cell grid, and the clouds' cells
 * are numbered one after another), so overlapping clouds do not interact.
 * Batching has no counterpart in the paper: one launch per stage serves many
 * small clouds that would each leave most of the GPU idle.
 *   cloud_offset int64 [nclouds+1] DEVICE: cloud_offset[0] = 0,
 *            cloud_offset[nclouds] = n, non-decreasing (empty clouds allowed);
 *            otherwise the status block records MAFP_EINVAL, col and order
 *            are not written and row_ptr is unspecified
 *   the other arguments as mafp_build_neighbours, indices global over all
 *   clouds.  cap_cells of the context bounds the sum of all clouds' cells.
 * nclouds outside [1, MAFP_MAX_CLOUDS] -> MAFP_EINVAL on the host.
 * mafp_build_neighbours is this call with nclouds = 1. */
int mafp_build_neighbours_batched(mafp_ctx *ctx, int64_t n, int32_t dtype, int32_t nclouds,
                                  const int64_t *cloud_offset, const void *pos_h,
                                  int64_t *row_ptr, int32_t *col, int64_t cap_nnz,
                                  int64_t *nnz_dev, int32_t *order, void *stream);

/* --------------------------------------------------------------------------
 * mafp_classify_pca -- model-transition detection of Sec. 4:
 *  3D wall particles: Alg. 2 -- resolution criterion (Sec. 4.1.1) over 3D
 *    neighbours j != i; with a free-surface neighbour, local PCA (Sec. 4.1.2,
 *    unweighted centroid and covariance of the 3D part of S_i, coordinates
 *    (x - x_i)/h_i), eps = 2 l3/(l1 + l2) < eps_lambda_max (Eq. EigenvalueLimit)
 *    and |n_i . w3| >= cos(theta*) (Eq. EigenvectorLimit, read as a maximum
 *    deviation), or a user request; only-wall neighbourhoods flag directly.
 *  2D particles: H_film of Eq. Height over the 2D part of S_i, flag when
 *    H_film >= h3D (Eq. 2Dto3Dcond) or on a user request; PCA gives the frame.
 *  then smoothing of Sec. 4.3 (no lone transitions, none right after one).
 *   pos_h x4, model/type/user/last uint8, normal x4 (inward unit normal),
 *   vol [n] (V_j of Eq. Height), h3d [n], row_ptr/col from build_neighbours.
 *   flag    uint8 [n] written: 0 stay, 1 -> 2D, 2 -> 3D (after smoothing)
 *   preflag uint8 [n] written: flags before smoothing (scratch the caller owns)
 *   eig     x4 [n] written: (l1, l2, l3, eps) for 3D wall and 2D particles, else 0
 *   frame   x4 [2n] written: (w1, 0), (w3, 0) per particle (same particles)
 *   hfilm   [n] written: Eq. Height for 2D particles, else 0
 *   near    uint8 [n] or NULL: 1 where a decision was within near_rel */
int mafp_classify_pca(mafp_ctx *ctx, int64_t n, int32_t dtype, const void *pos_h,
                      const uint8_t *model, const uint8_t *type, const void *normal,
                      const void *vol, const void *h3d, const uint8_t *user,
                      const uint8_t *last, const int64_t *row_ptr, const int32_t *col,
                      uint8_t *flag, uint8_t *preflag, void *eig, void *frame, void *hfilm,
                      uint8_t *near, void *stream);

/* --------------------------------------------------------------------------
 * mafp_build_stencils -- GFDM stencils of Eq. GFDM_Definition (Sec. 2.3,
 * consistency order 2) over the same-model part of S_i (Sec. 6.2):
 *  minimum-norm weighted least squares, c_ij = w_j p(q_j)^T lambda with
 *  (sum_j w_j p_j p_j^T) lambda = D p(0), W(s) = (e^{-a s^2} - e^{-a})/(1 - e^{-a})
 *  for s = |x_j - x_i|/h_i <= 1; 3D: 10 monomials of q = (x_j - x_i)/h_i;
 *  2D: 6 monomials of (xi, eta) in the tangent frame (w1, w3 x w1) of frame,
 *  the gradient returned in world coordinates c^xi t1 + c^eta t2.
 *   coef   x4 [nnz] written: (c^x, c^y, c^z, c^Lap) per CSR entry, 0 for
 *          entries of the other model and for deficient rows
 *   status uint8 [n] written: MAFP_STENCIL_*;  cond float [n] written:
 *          (max/min Cholesky pivot)^2, +inf for deficient rows. */
int mafp_build_stencils(mafp_ctx *ctx, int64_t n, int32_t dtype, const void *pos_h,
                        const uint8_t *model, const void *frame, const int64_t *row_ptr,
                        const int32_t *col, void *coef, uint8_t *status, float *cond,
                        void *stream);

/* --------------------------------------------------------------------------
 * mafp_build_stencils_noalloc -- mafp_build_stencils without a context and
 * without allocating (the paper has no counterpart: this serves callers).
 * Some callers cannot call cudaMalloc: a plug-in inside a host application
 * that owns the whole device-memory budget through its own pool, or a time
 * step that must not stall on the implicit device synchronisation of
 * cudaMalloc / cudaFree.  This entry point takes the same arrays as
 * mafp_build_stencils (plus the parameters, NULL = defaults) and uses, as its
 * only scratch, a fixed array compiled into the library: the FP64-retake queue
 * for up to MAFP_NOALLOC_MAX_PARTICLES particles plus a few counters, about
 * 4 MB, present on every GPU that loads the library until the process exits.
 *  - n > MAFP_NOALLOC_MAX_PARTICLES returns MAFP_ECAPACITY and enqueues nothing.
 *  - The first call on a device looks up the array's device address on the
 *    current device (cudaGetSymbolAddress); make that first call before any
 *    stream capture.  A failed lookup returns MAFP_ECUDA.
 *  - Every call shares the one array and resets the queue length itself, so
 *    calls whose work overlaps on the GPU (different streams, or host threads
 *    without ordering) race on it: serialise them.
 *  - Launch shapes are the defaults; device-side counters are not reported,
 *    and no error text is kept (there is no context to hold it): a failing
 *    CUDA call shows only as MAFP_ECUDA. */
#define MAFP_NOALLOC_MAX_PARTICLES (1 << 20)
int mafp_build_stencils_noalloc(int64_t n, int32_t dtype, const mafp_params *params,
                                const void *pos_h, const uint8_t *model, const void *frame,
                                const int64_t *row_ptr, const int32_t *col, void *coef,
                                uint8_t *status, float *cond, void *stream);

/* --------------------------------------------------------------------------
 * mafp_apply_ops -- stencil application, Eq. GFDM_Definition:
 *   out[i][f] = sum_{e in row i} coef[e] * (fields[col[e]][f] - fields[i][f]),
 *   f = u, v, w, p.  The coefficients must annihilate constants
 *   (sum_j c_ij = 0 for every operator), as the order-2 GFDM stencils of
 *   mafp_build_stencils do by construction; then this equals
 *   sum_j c_ij u_j, and forming u_j - u_i first removes the u_i sum_j c_ij
 *   residue that FP32 rounding of the coefficients would otherwise add.
 *   fields x4 [n];  out x4 [4n] written: out[4i+f] = (d_x, d_y, d_z, Lap) of field f */
int mafp_apply_ops(mafp_ctx *ctx, int64_t n, int32_t dtype, const int64_t *row_ptr,
                   const int32_t *col, const void *coef, const void *fields, void *out,
                   void *stream);

/* mafp_transpose_map -- for every CSR entry e = (i, j), the offset of i inside
 * row j (the sets are symmetric, Eq. Nbd), so transposed products gather
 * instead of scatter.  tloc uint16 [nnz] written; rows longer than 65535 give
 * MAFP_ECAPACITY in the status block. */
int mafp_transpose_map(mafp_ctx *ctx, int64_t n, const int64_t *row_ptr, const int32_t *col,
                       uint16_t *tloc, void *stream);

/* mafp_apply_ops_backward -- exact adjoint of mafp_apply_ops w.r.t. the
 * field values:  gfields[j][f] = sum_{i in S_j} sum_op coef_ij^op gout[4i+f][op]
 *                               - sum_op (sum_k coef_jk^op) gout[4j+f][op],
 * (the second term vanishes for stencils that annihilate constants).
 * tloc from mafp_transpose_map: every gfields[j] is gathered from row j in a
 * fixed order (deterministic).  tloc NULL: rows scatter into gfields with
 * atomic adds (no map needed; summation order unspecified, gfields zeroed by
 * the call).  gout x4 [4n], gfields x4 [n]. */
int mafp_apply_ops_backward(mafp_ctx *ctx, int64_t n, int32_t dtype, const int64_t *row_ptr,
                            const int32_t *col, const uint16_t *tloc, const void *coef,
                            const void *gout, void *gfields, void *stream);

/* mafp_build_stencils_backward -- adjoint of (build_stencils, apply_ops) with
 * respect to the particle positions, for a loss L that depends on
 * out = apply_ops(build_stencils(pos), fields) with gout = dL/dout:
 *   gpos[k] += sum over rows i and entries (i, j) of
 *              sum_op (sum_f gout[4i+f][op] fields[j][f]) d c_ij^op / d x_k,
 * recomputing the moment matrix and its Cholesky per particle (no stored
 * factors).  Neighbour sets and models are held fixed (piecewise constant).
 * Rows of 2D particles: `frame` must be the particle's local PCA frame
 * (Sec. 4.1.2) at these positions, as mafp_classify_pca writes it; its
 * dependence on the positions is included through the normal w3 (first-order
 * perturbation of the eigenvector of the scatter matrix, whose eigenvalues
 * are recomputed as Rayleigh quotients in the given frame); turning (w1, w2)
 * inside the plane changes no output and contributes nothing.  Rows whose
 * moment matrix is rank deficient contribute nothing.
 * gpos x4 [n] written (x, y, z, 0). */
int mafp_build_stencils_backward(mafp_ctx *ctx, int64_t n, int32_t dtype, const void *pos_h,
                                 const uint8_t *model, const void *frame,
                                 const int64_t *row_ptr, const int32_t *col,
                                 const void *fields, const void *gout, void *gpos,
                                 void *stream);

/* --------------------------------------------------------------------------
 * mafp_remap_switched -- model transition with data mapping, Sec. 5:
 *  flag 1 (3D -> 2D, Alg. 3): interior/free-surface 3D neighbours of flagged
 *   particles are candidates; each maps onto its nearest 3D wall particle in
 *   its own S_b (ties: lower index) when that one is flagged, and is deleted.
 *   The flagged particle averages v, p, rho, eta over itself and its set,
 *   sums mass, sets d^3 = 6m/(pi rho) and H = max |(x_b - x_i).n_i|, becomes 2D.
 *  flag 2 (2D -> 3D, Alg. 4): gamma = ceil(H / (c_psi h3D)) particles at
 *   x_i + k (H/gamma) n_i, k = 1..gamma (the last free surface, others
 *   interior), data copied, mass m/(1+gamma) each; the particle becomes a 3D wall.
 *  Survivors keep their relative order; added particles follow, by (i, k).
 *   row_ptr/col  the neighbourhoods S of Eq. Nbd from mafp_build_neighbours;
 *            the candidates are found from the rows of the flagged particles,
 *            which relies on S being symmetric (j in S_b exactly when b in S_j)
 *   in/out   mafp_state of device arrays (out capacity cap_out rows)
 *   old2new  int32 [n] written: new index or -1 when deleted
 *   n_out_dev int64 [1] written: particle count after the transition
 * If the result would exceed cap_out nothing is written to out and the
 * status block records MAFP_ECAPACITY with required = n_out. */
typedef struct {
  void *pos_h, *vp, *normal;                 /* x4 arrays: (x,y,z,h), (u,v,w,p), (n,0) */
  void *rho, *eta, *mass, *diam, *hfilm, *h3d; /* real arrays */
  uint8_t *model, *type, *last;
} mafp_state;

int mafp_remap_switched(mafp_ctx *ctx, int64_t n, int32_t dtype, const mafp_state *in,
                        const uint8_t *flag, const int64_t *row_ptr, const int32_t *col,
                        const mafp_state *out, int64_t cap_out, int32_t *old2new,
                        int64_t *n_out_dev, void *stream);

/* --------------------------------------------------------------------------
 * Kernel-level timing (no counterpart in the paper; a measurement aid).
 * mafp_profile(ctx, 1) clears the record and brackets every later kernel
 * launch of this context with CUDA events on its stream (up to 4096 launches);
 * mafp_profile(ctx, 0) stops recording.  mafp_profile_read synchronises the
 * device and writes up to cap entries aggregated by kernel name, returning
 * the number of entries in *count. */
typedef struct {
  char name[64];
  int64_t launches;
  double total_ms;
} mafp_kernel_time;

int mafp_profile(mafp_ctx *ctx, int32_t enable);
int mafp_profile_read(mafp_ctx *ctx, mafp_kernel_time *out, int32_t cap, int32_t *count);

/* --------------------------------------------------------------------------
 * Buffer zone of Sec. 5.3 (Alg. 5), in three calls around a transition of the
 * ghost cloud:
 *  mafp_ghost_sources -- first loop: src[i] = 1 when S_i (Eq. Nbd, all models;
 *    the distance h of Sec. 5.3 read as the neighbourhood) holds a particle of
 *    the other model, else 0.  src uint8 [n] written.
 *  mafp_ghost_seed -- second loop: every source is copied, in index order, as
 *    an intermediate ghost of the same model at the same place (last = 0);
 *    ghost_flag[g] is the transition it takes in the third loop (1: 3D wall
 *    -> 2D, 2: 2D -> 3D, 0: interior / free-surface 3D ghost, a candidate that
 *    Alg. 3 maps onto its nearest wall ghost); ghost_src[g] = its source
 *    index; *n_ghost_dev = the count.  If it exceeds cap_ghost nothing is
 *    copied and the status block records MAFP_ECAPACITY.
 *  third loop: mafp_build_neighbours over the n_ghost intermediate ghosts,
 *    then mafp_remap_switched with ghost_flag.
 *  mafp_ghost_append -- the ghosts that transition produced (last == 1; a
 *    candidate left without a wall ghost keeps its model and is dropped) are
 *    appended behind the n_regular particles already in `all`:
 *    *n_all_dev = n_regular + their count (MAFP_ECAPACITY above cap_all,
 *    nothing copied).  Stencils of the regular rows built over the union then
 *    use S_i plus the ghost neighbours of i's model (Eq. GhostDerivatives);
 *    no derivative is taken at a ghost. */
int mafp_ghost_sources(mafp_ctx *ctx, int64_t n, const uint8_t *model, const int64_t *row_ptr,
                       const int32_t *col, uint8_t *src, void *stream);
int mafp_ghost_seed(mafp_ctx *ctx, int64_t n, int32_t dtype, const mafp_state *in,
                    const uint8_t *src, const mafp_state *ghost, int64_t cap_ghost,
                    uint8_t *ghost_flag, int32_t *ghost_src, int64_t *n_ghost_dev, void *stream);
int mafp_ghost_append(mafp_ctx *ctx, int64_t n_regular, int64_t n_ghost, int32_t dtype,
                      const mafp_state *ghost, const mafp_state *all, int64_t cap_all,
                      int64_t *n_all_dev, void *stream);

/* --------------------------------------------------------------------------
 * mafp_film_momentum -- explicit update of the film model's momentum balance
 * (Eq. FilmMomentum, Sec. 2.2) for every 2D particle:
 *   v <- v + dt (-eta / (rho H^2) v - grad p / rho + g_par),  g_par = g - (g.n) n,
 * then v is projected onto the tangent plane (n = the particle's normal).
 * grad p is taken from `out` (mafp_apply_ops output x4 [4n]: out[4i+3] =
 * (d/dx, d/dy, d/dz, Lap) of field 3, the pressure slot of vp).  vp x4 [n] is
 * updated in place (u, v, w; p untouched); H = hfilm; particles with H <= 0
 * and 3D particles are left alone.  gravity: 3 doubles on the HOST. */
int mafp_film_momentum(mafp_ctx *ctx, int64_t n, int32_t dtype, const uint8_t *model, void *vp,
                       const void *rho, const void *eta, const void *hfilm, const void *normal,
                       const void *out, const double *gravity, double dt, void *stream);

/* mafp_plane_flux -- fluid volume through a plane over one step (Eq. InstFlux
 * times dt, Sec. 7.3, as a sum over crossing particles): a particle whose
 * signed distance to the plane (point, unit normal: 3 doubles each, HOST) goes
 * from < 0 at pos_old to >= 0 at pos_new adds its volume mass/rho, one going
 * back subtracts it.  acc_dev double [2] (DEVICE) accumulates (volume, number
 * of crossings); the caller zeroes it. */
int mafp_plane_flux(mafp_ctx *ctx, int64_t n, int32_t dtype, const void *pos_old,
                    const void *pos_new, const void *mass, const void *rho, const double *point,
                    const double *normal, double *acc_dev, void *stream);

/* mafp_normal_stress -- the wall-normal viscous stress of Sec. 7.3,
 * n^T S n = 2 eta n^T (grad v) n with S = eta (grad v + grad v^T), from the
 * applied gradients of the velocity fields (out[4i+a] = d v_a / d(x,y,z),
 * a = 0..2), summed over the particles with select[i] != 0:
 * acc_dev double [2] (DEVICE) accumulates (sum, count); the region average is
 * sum / count.  The caller zeroes acc_dev. */
int mafp_normal_stress(mafp_ctx *ctx, int64_t n, int32_t dtype, const uint8_t *select,
                       const void *out, const void *eta, const void *normal, double *acc_dev,
                       void *stream);

#ifdef __cplusplus
}
#endif
#endif
