/* oracle.h -- plain FP64 CPU oracle of the per-particle operator pipeline of
 * "Adaptive coupling of 3D and 2D fluid flow models" (Suchde, arXiv 2405.13165).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the CPU
 * baseline leg of the benchmark call this code.  It shares nothing with the
 * CUDA library (no headers, helpers or constants) and is written to be read
 * against the paper: every function names the section / equation it follows.
 *
 * Conventions (all arrays in caller particle order):
 *   P        double [n][4]   x, y, z, h  (h = support radius h_i of Eq. Nbd)
 *   model    uint8  [n]      0 = 3D bulk, 1 = 2D film
 *   type     uint8  [n]      0 = interior, 1 = free surface, 2 = wall (Sec. 2.3)
 *   normal   double [n][4]   inward unit wall normal n_i (Sec. 4.1.3, Sec. 5.2)
 *   row_ptr  int64  [n+1], col int32 [nnz]: neighbourhoods S_i in CSR form,
 *            rows ascending by particle index, i included (Eq. Nbd).
 */
#ifndef MAFP_ORACLE_H
#define MAFP_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
  double eps_lambda_max; /* Eq. EigenvalueLimit threshold, 0.15 in Sec. 4.1.2 */
  double theta_star;     /* Eq. EigenvectorLimit max deviation, pi/6 in Sec. 4.1.3 */
  double alpha_film;     /* alpha of Eq. Height (not given in the paper) */
  double alpha_w;        /* shape of the GFDM least-squares weight (not given) */
  double c_psi;          /* (r_min + r_max) / 2 of Sec. 5.2 (not given) */
  double near_rel;       /* relative band for reporting near-threshold decisions */
} orc_params;

typedef struct {
  double *pos_h, *vp, *normal;                       /* [.][4] */
  double *rho, *eta, *mass, *diam, *hfilm, *h3d;     /* [.] */
  uint8_t *model, *type, *last;                      /* [.] */
} orc_state;

/* Eq. Nbd membership test, written out. */
int orc_in_support(const double *P, int64_t i, int64_t j);
/* Row S_i by brute force over all n particles (the definition); returns |S_i|,
 * writes the ascending indices to out when out != NULL. */
int64_t orc_row_brute(int64_t n, const double *P, int64_t i, int32_t *out);
/* All rows via uniform cells of edge max_j h_j (every member of S_i lies in the
 * 27 cells around i).  Returns nnz; returns -1 (row_ptr still filled) when
 * nnz > cap_nnz. */
int64_t orc_neighbours(int64_t n, const double *P, int64_t *row_ptr, int32_t *col,
                       int64_t cap_nnz);

/* Symmetric 3x3 eigen-decomposition by cyclic Jacobi rotations; eigenvalues
 * descending in lam, unit eigenvectors as columns of V (V[r*3+k]). */
void orc_jacobi3(const double A[9], double lam[3], double V[9]);

/* Local PCA of Sec. 4.1.2 on the same-model part of S_i, in coordinates
 * q = (x - x_i)/h_i.  Returns n(S_i); lam descending, V columns w_1..w_3. */
int64_t orc_pca(const double *P, const uint8_t *model, const int64_t *row_ptr,
                const int32_t *col, int64_t i, double lam[3], double V[9]);

/* Detection of Sec. 4 (Alg. 2 for 3D wall particles, Eq. 2Dto3Dcond for film
 * particles) for the particles listed in rows (all when rows == NULL).
 * preflag: 0 stay, 1 -> 2D, 2 -> 3D.  eig[i] = (l1, l2, l3, eps_lambda),
 * frame[i] = (w1, 0, w3, 0), hfilm[i] = Eq. Height, near[i] = 1 when a decision
 * taken was within near_rel of its threshold. */
void orc_classify(int64_t n, const double *P, const uint8_t *model, const uint8_t *type,
                  const double *normal, const double *vol, const double *h3d,
                  const uint8_t *user, const int64_t *row_ptr, const int32_t *col,
                  const orc_params *prm, const int64_t *rows, int64_t nrows,
                  uint8_t *preflag, double *eig, double *frame, double *hfilm, uint8_t *near);

/* Space and time smoothing of Sec. 4.3 applied to pre-flags. */
void orc_smooth(int64_t n, const uint8_t *model, const uint8_t *preflag, const uint8_t *last,
                const int64_t *row_ptr, const int32_t *col, const int64_t *rows,
                int64_t nrows, uint8_t *flag);

/* GFDM stencils of Eq. GFDM_Definition (order 2) for the listed rows.
 * coef[e] = (c^x, c^y, c^z, c^Lap) for CSR entry e; status[i] 0 ok,
 * 1 rank deficient; cond[i] = (max/min Cholesky pivot)^2. */
void orc_stencils(int64_t n, const double *P, const uint8_t *model, const int64_t *row_ptr,
                  const int32_t *col, const orc_params *prm, const int64_t *rows,
                  int64_t nrows, double *coef, uint8_t *status, double *cond);

/* Gradient of a loss L(out) with respect to the positions x (gpos [n][4],
 * h component 0) through the stencils of orc_stencils, given
 * gout = dL/dout [n][4][4] and the fields; out_i = sum_j c_ij (u_j - u_i).
 * Neighbour sets and models are held fixed; film rows include the dependence
 * of their tangent frame (the local PCA of Sec. 4.1.2) on the positions. */
void orc_stencil_grad(int64_t n, const double *P, const uint8_t *model, const int64_t *row_ptr,
                      const int32_t *col, const orc_params *prm, const double *fields,
                      const double *gout, double *gpos);

/* Stencil application of Eq. GFDM_Definition: out[i][f] = (d_x, d_y, d_z, Lap)
 * of field f at particle i, fields f = 0..3. */
void orc_apply(int64_t n, const int64_t *row_ptr, const int32_t *col, const double *coef,
               const double *fields, const int64_t *rows, int64_t nrows, double *out);
/* Transpose of orc_apply: gfields[j][f] = sum_i sum_op coef_ij^op gout[i][f][op]. */
void orc_apply_T(int64_t n, const int64_t *row_ptr, const int32_t *col, const double *coef,
                 const double *gout, double *gfields);

/* Model transition of Sec. 5: Alg. 3 (flag 1, 3D -> 2D) and Alg. 4 (flag 2,
 * 2D -> 3D).  Survivors keep their order, new particles are appended.
 * Returns n_out, or -(n_out) when n_out > cap_out (nothing written). */
int64_t orc_remap(int64_t n, const orc_state *in, const uint8_t *flag, const int64_t *row_ptr,
                  const int32_t *col, const orc_params *prm, orc_state *out, int64_t cap_out,
                  int32_t *old2new);

/* Alg. 5, first loop: src[i] = 1 when S_i holds a particle of the other model. */
void orc_ghost_sources(int64_t n, const uint8_t *model, const int64_t *row_ptr,
                       const int32_t *col, uint8_t *src);

#ifdef __cplusplus
}
#endif

#endif
