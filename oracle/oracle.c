/* oracle.c -- plain FP64 CPU oracle of the per-particle operator pipeline of
 * "Adaptive coupling of 3D and 2D fluid flow models" (Suchde, arXiv 2405.13165).
 *
 * TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's CPU
 * baseline leg are its only callers.  Slow on purpose: every step is a plain
 * loop that can be checked against the paper by eye.  Built with
 * -ffp-contract=off so every product and sum rounds as written.
 *
 * Readings where the paper is silent or garbled (see the design notes):
 *   - Eq. Nbd is inclusive and evaluated on squares: d^2 <= ((h_i+h_j)/2)^2,
 *     d^2 = (dx*dx + dy*dy) + dz*dz, differences x_j - x_i.
 *   - Eq. EigenvectorLimit as printed (|n.w3| < cos theta*) contradicts
 *     "maximum deviation" and the cylinder result of Sec. 7.1; the test used
 *     is |n.w3| >= cos theta*.
 *   - Smoothing rule 1 (Sec. 4.3) counts a neighbour as "of the target model"
 *     when it already is, or is itself pre-flagged for the same target.
 *   - GFDM stencils (Sec. 2.3, Eq. GFDM_Definition): weighted least squares
 *     minimum-norm coefficients, quadratic basis, weight W of alpha_w.
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

enum { M3D = 0, M2D = 1 };
enum { T_INT = 0, T_FS = 1, T_WALL = 2 };
enum { USER_TO_2D = 1, USER_TO_3D = 2 };

/* ---------------------------------------------------------------------------
 * Neighbourhoods, Eq. Nbd (Sec. 2.2):  S_i = { j : |x_j - x_i| <= (h_i + h_j)/2 }.
 * ------------------------------------------------------------------------- */
static double dist2(const double *P, int64_t i, int64_t j) {
  double dx = P[4 * j + 0] - P[4 * i + 0];
  double dy = P[4 * j + 1] - P[4 * i + 1];
  double dz = P[4 * j + 2] - P[4 * i + 2];
  return (dx * dx + dy * dy) + dz * dz;
}

int orc_in_support(const double *P, int64_t i, int64_t j) {
  double r = (P[4 * i + 3] + P[4 * j + 3]) * 0.5;
  return dist2(P, i, j) <= r * r;
}

int64_t orc_row_brute(int64_t n, const double *P, int64_t i, int32_t *out) {
  int64_t k = 0;
  for (int64_t j = 0; j < n; ++j)
    if (orc_in_support(P, i, j)) {
      if (out) out[k] = (int32_t)j;
      ++k;
    }
  return k;
}

typedef struct {
  int64_t key;
  int64_t idx;
} keyidx;

static int cmp_keyidx(const void *a, const void *b) {
  const keyidx *x = (const keyidx *)a, *y = (const keyidx *)b;
  if (x->key != y->key) return x->key < y->key ? -1 : 1;
  return x->idx < y->idx ? -1 : (x->idx > y->idx);
}

static int cmp_i32(const void *a, const void *b) {
  int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
  return x < y ? -1 : (x > y);
}

/* first position in sorted cells[0..n) with key >= k */
static int64_t lower_key(const keyidx *cells, int64_t n, int64_t k) {
  int64_t lo = 0, hi = n;
  while (lo < hi) {
    int64_t mid = lo + (hi - lo) / 2;
    if (cells[mid].key < k) lo = mid + 1; else hi = mid;
  }
  return lo;
}

typedef struct {
  double lo[3], c;
  int64_t dim[3];
} grid3;

static void cell_of(const grid3 *g, const double *p, int64_t cc[3]) {
  for (int a = 0; a < 3; ++a) {
    int64_t v = (int64_t)floor((p[a] - g->lo[a]) / g->c);
    if (v < 0) v = 0;
    if (v >= g->dim[a]) v = g->dim[a] - 1;
    cc[a] = v;
  }
}

/* Members of S_i from the 27 cells around i (cells of edge max h, so the
 * radius (h_i+h_j)/2 never reaches beyond them), sorted ascending. */
static int64_t row_grid(const grid3 *g, const keyidx *cells, int64_t n, const double *P,
                        int64_t i, int32_t *out) {
  int64_t cc[3], k = 0;
  cell_of(g, P + 4 * i, cc);
  for (int64_t dz = -1; dz <= 1; ++dz)
    for (int64_t dy = -1; dy <= 1; ++dy)
      for (int64_t dx = -1; dx <= 1; ++dx) {
        int64_t x = cc[0] + dx, y = cc[1] + dy, z = cc[2] + dz;
        if (x < 0 || y < 0 || z < 0 || x >= g->dim[0] || y >= g->dim[1] || z >= g->dim[2])
          continue;
        int64_t key = (z * g->dim[1] + y) * g->dim[0] + x;
        for (int64_t s = lower_key(cells, n, key); s < n && cells[s].key == key; ++s) {
          int64_t j = cells[s].idx;
          if (orc_in_support(P, i, j)) {
            if (out) out[k] = (int32_t)j;
            ++k;
          }
        }
      }
  if (out) qsort(out, (size_t)k, sizeof(int32_t), cmp_i32);
  return k;
}

int64_t orc_neighbours(int64_t n, const double *P, int64_t *row_ptr, int32_t *col,
                       int64_t cap_nnz) {
  row_ptr[0] = 0;
  if (n <= 0) return 0;
  grid3 g;
  double hi[3];
  g.c = 0.0;
  for (int a = 0; a < 3; ++a) g.lo[a] = hi[a] = P[a];
  for (int64_t i = 0; i < n; ++i) {
    for (int a = 0; a < 3; ++a) {
      if (P[4 * i + a] < g.lo[a]) g.lo[a] = P[4 * i + a];
      if (P[4 * i + a] > hi[a]) hi[a] = P[4 * i + a];
    }
    if (P[4 * i + 3] > g.c) g.c = P[4 * i + 3];
  }
  if (!(g.c > 0.0)) g.c = 1.0;
  for (int a = 0; a < 3; ++a) g.dim[a] = (int64_t)floor((hi[a] - g.lo[a]) / g.c) + 1;
  keyidx *cells = (keyidx *)malloc(sizeof(keyidx) * (size_t)n);
  for (int64_t i = 0; i < n; ++i) {
    int64_t cc[3];
    cell_of(&g, P + 4 * i, cc);
    cells[i].key = (cc[2] * g.dim[1] + cc[1]) * g.dim[0] + cc[0];
    cells[i].idx = i;
  }
  qsort(cells, (size_t)n, sizeof(keyidx), cmp_keyidx);
#pragma omp parallel for schedule(dynamic, 256)
  for (int64_t i = 0; i < n; ++i) row_ptr[i + 1] = row_grid(&g, cells, n, P, i, NULL);
  for (int64_t i = 0; i < n; ++i) row_ptr[i + 1] += row_ptr[i];
  int64_t nnz = row_ptr[n];
  if (nnz > cap_nnz || col == NULL) {
    free(cells);
    return nnz > cap_nnz ? -1 : nnz;
  }
#pragma omp parallel for schedule(dynamic, 256)
  for (int64_t i = 0; i < n; ++i) row_grid(&g, cells, n, P, i, col + row_ptr[i]);
  free(cells);
  return nnz;
}

/* ---------------------------------------------------------------------------
 * Symmetric 3x3 eigen-decomposition (cyclic Jacobi, textbook form):
 * repeatedly apply plane rotations J(p,q,c,s) chosen so that (J^T A J)_pq = 0.
 * ------------------------------------------------------------------------- */
static void matmul3(const double A[9], const double B[9], double C[9]) {
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) {
      double s = 0.0;
      for (int k = 0; k < 3; ++k) s += A[r * 3 + k] * B[k * 3 + c];
      C[r * 3 + c] = s;
    }
}

void orc_jacobi3(const double Ain[9], double lam[3], double V[9]) {
  double A[9], T[9], J[9], Jt[9];
  memcpy(A, Ain, sizeof(A));
  for (int k = 0; k < 9; ++k) V[k] = (k % 4 == 0) ? 1.0 : 0.0;
  double tot = 0.0;
  for (int k = 0; k < 9; ++k) tot += A[k] * A[k];
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = A[1] * A[1] + A[2] * A[2] + A[5] * A[5];
    if (off <= 1e-40 * tot || off == 0.0) break;
    static const int PQ[3][2] = {{0, 1}, {0, 2}, {1, 2}};
    for (int r = 0; r < 3; ++r) {
      int p = PQ[r][0], q = PQ[r][1];
      double apq = A[p * 3 + q];
      if (apq == 0.0) continue;
      double tau = (A[q * 3 + q] - A[p * 3 + p]) / (2.0 * apq);
      double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
      double c = 1.0 / sqrt(1.0 + t * t), s = t * c;
      for (int k = 0; k < 9; ++k) J[k] = (k % 4 == 0) ? 1.0 : 0.0;
      J[p * 3 + p] = c;
      J[p * 3 + q] = s;
      J[q * 3 + p] = -s;
      J[q * 3 + q] = c;
      for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) Jt[a * 3 + b] = J[b * 3 + a];
      matmul3(Jt, A, T);
      matmul3(T, J, A);
      A[p * 3 + q] = A[q * 3 + p] = 0.0;
      matmul3(V, J, T);
      memcpy(V, T, sizeof(T));
    }
  }
  /* sort descending (eigenvectors follow) */
  int ord[3] = {0, 1, 2};
  for (int a = 0; a < 3; ++a)
    for (int b = a + 1; b < 3; ++b)
      if (A[ord[b] * 4] > A[ord[a] * 4]) {
        int t = ord[a]; ord[a] = ord[b]; ord[b] = t;
      }
  double W[9];
  for (int k = 0; k < 3; ++k) {
    lam[k] = A[ord[k] * 4];
    for (int r = 0; r < 3; ++r) W[r * 3 + k] = V[r * 3 + ord[k]];
  }
  memcpy(V, W, sizeof(W));
}

/* ---------------------------------------------------------------------------
 * Local PCA, Sec. 4.1.2:  P_i = sum_{j in S_i} (x_j - x_c)(x_j - x_c)^T with the
 * unweighted centroid x_c = (1/n(S_i)) sum_j x_j, over the same-model part of
 * S_i (each model keeps its own search structure, Sec. 5).  Coordinates are
 * shifted by x_i and divided by h_i, which scales every eigenvalue by 1/h_i^2
 * and leaves ratios and eigenvectors unchanged.
 * ------------------------------------------------------------------------- */
static int64_t pca_scatter(const double *P, const uint8_t *model, const int64_t *row_ptr,
                           const int32_t *col, int64_t i, double yc[3], double C[9]) {
  double h = P[4 * i + 3];
  int64_t m = 0;
  for (int a = 0; a < 3; ++a) yc[a] = 0.0;
  for (int k = 0; k < 9; ++k) C[k] = 0.0;
  for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
    int64_t j = col[e];
    if (model[j] != model[i]) continue;
    for (int a = 0; a < 3; ++a) yc[a] += (P[4 * j + a] - P[4 * i + a]) / h;
    ++m;
  }
  if (m > 0) {
    for (int a = 0; a < 3; ++a) yc[a] /= (double)m;
    for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
      int64_t j = col[e];
      if (model[j] != model[i]) continue;
      double d[3];
      for (int a = 0; a < 3; ++a) d[a] = (P[4 * j + a] - P[4 * i + a]) / h - yc[a];
      for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) C[a * 3 + b] += d[a] * d[b];
    }
  }
  return m;
}

int64_t orc_pca(const double *P, const uint8_t *model, const int64_t *row_ptr,
                const int32_t *col, int64_t i, double lam[3], double V[9]) {
  double yc[3], C[9];
  int64_t m = pca_scatter(P, model, row_ptr, col, i, yc, C);
  orc_jacobi3(C, lam, V);
  return m;
}

/* ---------------------------------------------------------------------------
 * Detection, Sec. 4.
 * ------------------------------------------------------------------------- */
static int near_rel(double v, double thr, double rel) {
  return fabs(v - thr) <= rel * fabs(thr);
}

static void classify_one(int64_t i, const double *P, const uint8_t *model, const uint8_t *type,
                         const double *normal, const double *vol, const double *h3d,
                         const uint8_t *user, const int64_t *row_ptr, const int32_t *col,
                         const orc_params *prm, uint8_t *preflag, double *eig, double *frame,
                         double *hfilm, uint8_t *near) {
  uint8_t pre = 0, nr = 0;
  double lam[3] = {0, 0, 0}, V[9] = {0}, eps = INFINITY, H = 0.0;
  int did_pca = 0;
  if (model[i] == M3D) {
    if (type[i] == T_WALL) {
      /* Sec. 4.1.1 resolution criterion over the 3D neighbours j != i. */
      int has_fs = 0, has_int = 0;
      for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
        int64_t j = col[e];
        if (j == i || model[j] != M3D) continue;
        if (type[j] == T_FS) has_fs = 1;
        if (type[j] == T_INT) has_int = 1;
      }
      orc_pca(P, model, row_ptr, col, i, lam, V);
      did_pca = 1;
      eps = (lam[0] + lam[1]) > 0.0 ? 2.0 * lam[2] / (lam[0] + lam[1]) : INFINITY;
      if (has_fs) {
        /* Alg. 2: PCA criteria (Eq. EigenvalueLimit, Eq. EigenvectorLimit)
         * or a user-defined criterion, both inside the resolution branch. */
        double ndw = fabs(normal[4 * i] * V[2] + normal[4 * i + 1] * V[5] +
                          normal[4 * i + 2] * V[8]);
        double cth = cos(prm->theta_star);
        int pca_ok = (eps < prm->eps_lambda_max) && (ndw >= cth);
        if (pca_ok || (user[i] & USER_TO_2D)) pre = 1;
        if (!(user[i] & USER_TO_2D)) {
          int eps_near = near_rel(eps, prm->eps_lambda_max, prm->near_rel);
          int ang_near = fabs(ndw - cth) <= prm->near_rel;
          /* w3 is not unique when l2 = l3 (e.g. collinear neighbours): the
           * eigenvector test has no single answer and is reported instead */
          int degenerate = (lam[1] - lam[2]) <= 1e-9 * lam[0];
          /* a near-threshold quantity only matters when the other test passes */
          if ((eps_near && ndw >= cth) || (ang_near && eps < prm->eps_lambda_max) ||
              (eps_near && ang_near) || (degenerate && eps < prm->eps_lambda_max))
            nr = 1;
        }
      } else if (!has_int) {
        pre = 1; /* only wall neighbours (or none): h_i >> H_film */
      }
    }
  } else {
    /* Eq. Height over the 2D part of S_i, then Eq. 2Dto3Dcond. */
    for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
      int64_t j = col[e];
      if (model[j] != M2D) continue;
      double hj = P[4 * j + 3];
      double d2 = dist2(P, i, j);
      H += prm->alpha_film / (M_PI * hj * hj) * exp(-prm->alpha_film * d2 / (hj * hj)) * vol[j];
    }
    if (H >= h3d[i] || (user[i] & USER_TO_3D)) pre = 2;
    if (!(user[i] & USER_TO_3D) && near_rel(H, h3d[i], prm->near_rel)) nr = 1;
    orc_pca(P, model, row_ptr, col, i, lam, V);
    did_pca = 1;
    eps = (lam[0] + lam[1]) > 0.0 ? 2.0 * lam[2] / (lam[0] + lam[1]) : INFINITY;
  }
  preflag[i] = pre;
  if (near) near[i] = nr;
  if (hfilm) hfilm[i] = H;
  if (eig) {
    eig[4 * i + 0] = lam[0];
    eig[4 * i + 1] = lam[1];
    eig[4 * i + 2] = lam[2];
    eig[4 * i + 3] = did_pca ? eps : 0.0;
  }
  if (frame) {
    for (int a = 0; a < 3; ++a) {
      frame[8 * i + a] = did_pca ? V[a * 3 + 0] : 0.0;
      frame[8 * i + 4 + a] = did_pca ? V[a * 3 + 2] : 0.0;
    }
    frame[8 * i + 3] = 0.0;
    frame[8 * i + 7] = 0.0;
  }
}

void orc_classify(int64_t n, const double *P, const uint8_t *model, const uint8_t *type,
                  const double *normal, const double *vol, const double *h3d,
                  const uint8_t *user, const int64_t *row_ptr, const int32_t *col,
                  const orc_params *prm, const int64_t *rows, int64_t nrows,
                  uint8_t *preflag, double *eig, double *frame, double *hfilm, uint8_t *near) {
  int64_t cnt = rows ? nrows : n;
#pragma omp parallel for schedule(dynamic, 64)
  for (int64_t r = 0; r < cnt; ++r) {
    int64_t i = rows ? rows[r] : r;
    classify_one(i, P, model, type, normal, vol, h3d, user, row_ptr, col, prm, preflag, eig,
                 frame, hfilm, near);
  }
}

/* Sec. 4.3: (1) no transition when no other neighbour is of (or is already
 * flagged for) the target model; (2) no transition right after a transition. */
void orc_smooth(int64_t n, const uint8_t *model, const uint8_t *preflag, const uint8_t *last,
                const int64_t *row_ptr, const int32_t *col, const int64_t *rows,
                int64_t nrows, uint8_t *flag) {
  int64_t cnt = rows ? nrows : n;
#pragma omp parallel for schedule(dynamic, 256)
  for (int64_t r = 0; r < cnt; ++r) {
    int64_t i = rows ? rows[r] : r;
    uint8_t f = preflag[i];
    if (f != 0 && last[i]) f = 0;
    if (f != 0) {
      uint8_t target = (f == 1) ? M2D : M3D;
      int ok = 0;
      for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
        int64_t j = col[e];
        if (j == i) continue;
        if (model[j] == target || preflag[j] == preflag[i]) ok = 1;
      }
      if (!ok) f = 0;
    }
    flag[i] = f;
  }
}

/* ---------------------------------------------------------------------------
 * GFDM stencils, Sec. 2.3 and Eq. GFDM_Definition (consistency order 2: every
 * monomial of degree <= 2 is differentiated exactly).  Coefficients are the
 * minimum of sum_j c_j^2 / w_j subject to the moment conditions
 * sum_j c_j p(q_j) = D p(0), i.e. c_j = w_j p(q_j)^T lambda with
 * (sum_j w_j p_j p_j^T) lambda = D p(0).
 * ------------------------------------------------------------------------- */
static double weight_w(double s, double alpha) {
  if (s > 1.0) return 0.0;
  double ea = exp(-alpha);
  return (exp(-alpha * s * s) - ea) / (1.0 - ea);
}

/* Cholesky A = L L^T of an m x m SPD matrix (row-major, lower part used).
 * Returns 0, or 1 when a pivot is <= tol (rank deficient). */
static int cholesky(int m, double *A, double tol, double *pmin, double *pmax) {
  *pmin = INFINITY;
  *pmax = 0.0;
  for (int k = 0; k < m; ++k) {
    double d = A[k * m + k];
    for (int l = 0; l < k; ++l) d -= A[k * m + l] * A[k * m + l];
    if (!(d > tol)) return 1;
    double Lkk = sqrt(d);
    A[k * m + k] = Lkk;
    if (Lkk < *pmin) *pmin = Lkk;
    if (Lkk > *pmax) *pmax = Lkk;
    for (int r = k + 1; r < m; ++r) {
      double s = A[r * m + k];
      for (int l = 0; l < k; ++l) s -= A[r * m + l] * A[k * m + l];
      A[r * m + k] = s / Lkk;
    }
  }
  return 0;
}

static void chol_solve(int m, const double *L, const double *b, double *x) {
  double y[16];
  for (int r = 0; r < m; ++r) {
    double s = b[r];
    for (int l = 0; l < r; ++l) s -= L[r * m + l] * y[l];
    y[r] = s / L[r * m + r];
  }
  for (int r = m - 1; r >= 0; --r) {
    double s = y[r];
    for (int l = r + 1; l < m; ++l) s -= L[l * m + r] * x[l];
    x[r] = s / L[r * m + r];
  }
}

static void basis3(const double q[3], double p[10]) {
  p[0] = 1.0;
  p[1] = q[0]; p[2] = q[1]; p[3] = q[2];
  p[4] = q[0] * q[0]; p[5] = q[1] * q[1]; p[6] = q[2] * q[2];
  p[7] = q[0] * q[1]; p[8] = q[0] * q[2]; p[9] = q[1] * q[2];
}

static void basis2(double xi, double eta, double p[6]) {
  p[0] = 1.0; p[1] = xi; p[2] = eta;
  p[3] = xi * xi; p[4] = xi * eta; p[5] = eta * eta;
}

static void stencil_one(int64_t i, const double *P, const uint8_t *model,
                        const int64_t *row_ptr, const int32_t *col, const orc_params *prm,
                        double *coef, uint8_t *status, double *cond) {
  const int is2d = model[i] == M2D;
  const int m = is2d ? 6 : 10;
  const double h = P[4 * i + 3];
  double t1[3] = {0, 0, 0}, t2[3] = {0, 0, 0};
  if (is2d) {
    /* tangent frame of the film from the local PCA (w1, w2 span the surface) */
    double lam[3], V[9];
    orc_pca(P, model, row_ptr, col, i, lam, V);
    for (int a = 0; a < 3; ++a) { t1[a] = V[a * 3 + 0]; t2[a] = V[a * 3 + 1]; }
  }
  double A[100] = {0}, p[10];
  int64_t cnt = 0;
  for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
    int64_t j = col[e];
    for (int k = 0; k < 4; ++k) coef[4 * e + k] = 0.0;
    if (model[j] != model[i]) continue;
    double d[3], q[3];
    for (int a = 0; a < 3; ++a) d[a] = P[4 * j + a] - P[4 * i + a];
    double w = weight_w(sqrt(dist2(P, i, j)) / h, prm->alpha_w);
    if (is2d) {
      basis2((d[0] * t1[0] + d[1] * t1[1] + d[2] * t1[2]) / h,
             (d[0] * t2[0] + d[1] * t2[1] + d[2] * t2[2]) / h, p);
    } else {
      for (int a = 0; a < 3; ++a) q[a] = d[a] / h;
      basis3(q, p);
    }
    for (int r = 0; r < m; ++r)
      for (int c = 0; c < m; ++c) A[r * m + c] += w * p[r] * p[c];
    ++cnt;
  }
  double tr = 0.0;
  for (int r = 0; r < m; ++r) tr += A[r * m + r];
  double pmin, pmax;
  if (cnt < m || cholesky(m, A, 1e-12 * tr, &pmin, &pmax)) {
    status[i] = 1;
    cond[i] = INFINITY;
    return;
  }
  status[i] = 0;
  cond[i] = (pmax / pmin) * (pmax / pmin);
  /* right-hand sides: derivatives of the basis at the particle (q = 0) */
  double b[4][10] = {{0}}, lam[4][10];
  if (is2d) {
    b[0][1] = 1.0 / h;                          /* d/dxi   */
    b[1][2] = 1.0 / h;                          /* d/deta  */
    b[2][3] = 2.0 / (h * h); b[2][5] = 2.0 / (h * h); /* Laplacian in the plane */
    for (int k = 0; k < 3; ++k) chol_solve(m, A, b[k], lam[k]);
  } else {
    b[0][1] = 1.0 / h;
    b[1][2] = 1.0 / h;
    b[2][3] = 1.0 / h;
    b[3][4] = 2.0 / (h * h); b[3][5] = 2.0 / (h * h); b[3][6] = 2.0 / (h * h);
    for (int k = 0; k < 4; ++k) chol_solve(m, A, b[k], lam[k]);
  }
  for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
    int64_t j = col[e];
    if (model[j] != model[i]) continue;
    double d[3], q[3];
    for (int a = 0; a < 3; ++a) d[a] = P[4 * j + a] - P[4 * i + a];
    double w = weight_w(sqrt(dist2(P, i, j)) / h, prm->alpha_w);
    if (is2d) {
      basis2((d[0] * t1[0] + d[1] * t1[1] + d[2] * t1[2]) / h,
             (d[0] * t2[0] + d[1] * t2[1] + d[2] * t2[2]) / h, p);
      double c[3];
      for (int k = 0; k < 3; ++k) {
        double s = 0.0;
        for (int r = 0; r < m; ++r) s += p[r] * lam[k][r];
        c[k] = w * s;
      }
      /* tangential gradient in world coordinates: c^xi t1 + c^eta t2 */
      for (int a = 0; a < 3; ++a) coef[4 * e + a] = c[0] * t1[a] + c[1] * t2[a];
      coef[4 * e + 3] = c[2];
    } else {
      for (int a = 0; a < 3; ++a) q[a] = d[a] / h;
      basis3(q, p);
      for (int k = 0; k < 4; ++k) {
        double s = 0.0;
        for (int r = 0; r < m; ++r) s += p[r] * lam[k][r];
        coef[4 * e + k] = w * s;
      }
    }
  }
}

void orc_stencils(int64_t n, const double *P, const uint8_t *model, const int64_t *row_ptr,
                  const int32_t *col, const orc_params *prm, const int64_t *rows,
                  int64_t nrows, double *coef, uint8_t *status, double *cond) {
  int64_t cnt = rows ? nrows : n;
#pragma omp parallel for schedule(dynamic, 64)
  for (int64_t r = 0; r < cnt; ++r) {
    int64_t i = rows ? rows[r] : r;
    stencil_one(i, P, model, row_ptr, col, prm, coef, status, cond);
  }
}

/* ---------------------------------------------------------------------------
 * Adjoint of the stencils with respect to the positions (differentiation of
 * out_i = sum_j c_ij (u_j - u_i), Eq. GFDM_Definition, with the stencils of
 * stencil_one).  For one row, with gbar_jk = dL/dc_jk:
 *   lambda_k = A^-1 b_k,  lbar_k = sum_j gbar_jk w_j p_j,  mu_k = A^-1 lbar_k,
 *   s_jk = p_j.lambda_k,  t_jk = p_j.mu_k,
 *   wbar_j = sum_k (gbar_jk - t_jk) s_jk,
 *   pbar_j = w_j sum_k (gbar_jk lambda_k - s_jk mu_k - t_jk lambda_k),
 * then through p(q) and w(|q|) to q_j = (x_j - x_i)/h_i.  Neighbour sets and
 * models are held fixed (piecewise constant in the positions).
 *
 * Film rows also depend on the positions through their tangent frame, the
 * local PCA of Sec. 4.1.2 that stencil_one recomputes: t1 = w1, t2 = w2 of the
 * scatter matrix Ps = sum_j z_j z_j^T, z_j = y_j - y_c, y_j = (x_j - x_i)/h_i,
 * y_c the centroid.  The outputs (tangential gradient c^xi t1 + c^eta t2 and
 * the plane Laplacian) do not change when (t1, t2) turn inside the plane, so
 * only the normal n = w3 matters.  With tbar_k = dL/dt_k at fixed n, turning
 * the frame with n (dt_k = -n (t_k . dn)) gives dL = -sum_k (tbar_k . n)(t_k . dn);
 * first-order perturbation of the eigenvector w3,
 *   dn = -sum_{k=1,2} w_k (w_k^T dPs n) / (l_k - l3),
 * and dPs = sum_j (dy_j z_j^T + z_j dy_j^T) (the centroid terms cancel since
 * sum_j z_j = 0) give
 *   ybar_j = sum_k beta_k (t_k (n . z_j) + n (t_k . z_j)),
 *   beta_k = (tbar_k . n) / (l_k - l3),
 * passed to x_j and x_i like the stencil terms.
 * ------------------------------------------------------------------------- */
static double weight_dw_over_s(double s, double alpha) {
  /* W'(s)/s for s <= 1 (W of weight_w), 0 outside the support */
  if (s > 1.0) return 0.0;
  return -2.0 * alpha * exp(-alpha * s * s) / (1.0 - exp(-alpha));
}

static double dot3(const double a[3], const double b[3]) {
  return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}

static void stencil_grad_one(int64_t i, const double *P, const uint8_t *model,
                             const int64_t *row_ptr, const int32_t *col, const orc_params *prm,
                             const double *fields, const double *gout, double *gpos) {
  const int is2d = model[i] == M2D;
  const int m = is2d ? 6 : 10, nr = is2d ? 3 : 4;
  const double h = P[4 * i + 3];
  double t1[3] = {0, 0, 0}, t2[3] = {0, 0, 0}, nv[3] = {0, 0, 0};
  double plam[3] = {0, 0, 0}, yc[3] = {0, 0, 0};
  if (is2d) {
    double V[9], Ps[9];
    pca_scatter(P, model, row_ptr, col, i, yc, Ps);
    orc_jacobi3(Ps, plam, V);
    for (int a = 0; a < 3; ++a) {
      t1[a] = V[a * 3 + 0];
      t2[a] = V[a * 3 + 1];
      nv[a] = V[a * 3 + 2];
    }
  }
  double A[100] = {0}, p[10];
  int64_t cnt = 0;
  for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
    int64_t j = col[e];
    if (model[j] != model[i]) continue;
    double d[3], q[3];
    for (int a = 0; a < 3; ++a) d[a] = P[4 * j + a] - P[4 * i + a];
    double w = weight_w(sqrt(dist2(P, i, j)) / h, prm->alpha_w);
    if (is2d) {
      basis2(dot3(d, t1) / h, dot3(d, t2) / h, p);
    } else {
      for (int a = 0; a < 3; ++a) q[a] = d[a] / h;
      basis3(q, p);
    }
    for (int r = 0; r < m; ++r)
      for (int c = 0; c < m; ++c) A[r * m + c] += w * p[r] * p[c];
    ++cnt;
  }
  double tr = 0.0;
  for (int r = 0; r < m; ++r) tr += A[r * m + r];
  double pmin, pmax;
  if (cnt < m || cholesky(m, A, 1e-12 * tr, &pmin, &pmax)) return; /* zero stencil, no gradient */
  double b[4][10] = {{0}}, lam[4][10], lbar[4][10] = {{0}}, mu[4][10];
  if (is2d) {
    b[0][1] = 1.0 / h; b[1][2] = 1.0 / h;
    b[2][3] = 2.0 / (h * h); b[2][5] = 2.0 / (h * h);
  } else {
    b[0][1] = 1.0 / h; b[1][2] = 1.0 / h; b[2][3] = 1.0 / h;
    b[3][4] = 2.0 / (h * h); b[3][5] = 2.0 / (h * h); b[3][6] = 2.0 / (h * h);
  }
  for (int k = 0; k < nr; ++k) chol_solve(m, A, b[k], lam[k]);
  /* dL/dt_k of a film row at fixed n, summed over the row */
  double tbar[2][3] = {{0, 0, 0}, {0, 0, 0}};
  /* dL/dc for the row: gbar_jk = sum_f gout[i][f][op] (u_j - u_i); for a film row
   * the gradient outputs are c^xi t1 + c^eta t2, so gbar^xi = gbar . t1, etc. */
  for (int pass = 0; pass < 2; ++pass) {
    for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
      int64_t j = col[e];
      if (model[j] != model[i]) continue;
      double g4[4];
      for (int op = 0; op < 4; ++op) {
        double s = 0.0;
        for (int f = 0; f < 4; ++f) s += gout[16 * i + 4 * f + op] * (fields[4 * j + f] - fields[4 * i + f]);
        g4[op] = s;
      }
      double gb[4];
      if (is2d) {
        gb[0] = dot3(g4, t1);
        gb[1] = dot3(g4, t2);
        gb[2] = g4[3];
      } else {
        for (int k = 0; k < 4; ++k) gb[k] = g4[k];
      }
      double d[3], q[3];
      for (int a = 0; a < 3; ++a) d[a] = P[4 * j + a] - P[4 * i + a];
      double s_ = sqrt(dist2(P, i, j)) / h;
      double w = weight_w(s_, prm->alpha_w);
      double xi = 0, eta = 0;
      if (is2d) {
        xi = dot3(d, t1) / h;
        eta = dot3(d, t2) / h;
        basis2(xi, eta, p);
      } else {
        for (int a = 0; a < 3; ++a) q[a] = d[a] / h;
        basis3(q, p);
      }
      if (pass == 0) {
        for (int k = 0; k < nr; ++k)
          for (int r = 0; r < m; ++r) lbar[k][r] += gb[k] * w * p[r];
        continue;
      }
      double sk[4], tk[4], wbar = 0.0, pbar[10] = {0};
      for (int k = 0; k < nr; ++k) {
        sk[k] = 0.0;
        tk[k] = 0.0;
        for (int r = 0; r < m; ++r) {
          sk[k] += p[r] * lam[k][r];
          tk[k] += p[r] * mu[k][r];
        }
        wbar += (gb[k] - tk[k]) * sk[k];
        for (int r = 0; r < m; ++r)
          pbar[r] += w * (gb[k] * lam[k][r] - sk[k] * mu[k][r] - tk[k] * lam[k][r]);
      }
      double dbar[3];
      double wq = weight_dw_over_s(s_, prm->alpha_w) * wbar; /* dW/dq = W'(s) q / s */
      if (is2d) {
        double xib = pbar[1] + 2.0 * xi * pbar[3] + eta * pbar[4];
        double etb = pbar[2] + xi * pbar[4] + 2.0 * eta * pbar[5];
        for (int a = 0; a < 3; ++a) dbar[a] = (xib * t1[a] + etb * t2[a]) / h + wq * d[a] / (h * h);
        /* the frame enters through xi = d.t1/h, eta = d.t2/h and through the
         * world-coordinate gradient c^xi t1 + c^eta t2 (c^xi = w s_0, c^eta = w s_1) */
        for (int a = 0; a < 3; ++a) {
          tbar[0][a] += xib * d[a] / h + g4[a] * w * sk[0];
          tbar[1][a] += etb * d[a] / h + g4[a] * w * sk[1];
        }
      } else {
        double qb[3];
        qb[0] = pbar[1] + 2.0 * q[0] * pbar[4] + q[1] * pbar[7] + q[2] * pbar[8];
        qb[1] = pbar[2] + 2.0 * q[1] * pbar[5] + q[0] * pbar[7] + q[2] * pbar[9];
        qb[2] = pbar[3] + 2.0 * q[2] * pbar[6] + q[0] * pbar[8] + q[1] * pbar[9];
        for (int a = 0; a < 3; ++a) dbar[a] = (qb[a] + wq * q[a]) / h;
      }
      for (int a = 0; a < 3; ++a) {
        gpos[4 * j + a] += dbar[a];
        gpos[4 * i + a] -= dbar[a];
      }
    }
    if (pass == 0)
      for (int k = 0; k < nr; ++k) chol_solve(m, A, lbar[k], mu[k]);
  }
  if (!is2d) return;
  /* film frame: through n = w3 of the local PCA to the scaled positions y_j.
   * A gap l_k - l3 of zero leaves w3 undefined: no term is taken then. */
  double beta[2];
  for (int k = 0; k < 2; ++k) {
    double gap = plam[k] - plam[2];
    beta[k] = gap > 0.0 ? dot3(tbar[k], nv) / gap : 0.0;
  }
  const double *tk_[2] = {t1, t2};
  for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
    int64_t j = col[e];
    if (model[j] != model[i]) continue;
    double z[3], ybar[3] = {0, 0, 0};
    for (int a = 0; a < 3; ++a) z[a] = (P[4 * j + a] - P[4 * i + a]) / h - yc[a];
    double nz = dot3(nv, z);
    for (int k = 0; k < 2; ++k) {
      double tz = dot3(tk_[k], z);
      for (int a = 0; a < 3; ++a) ybar[a] += beta[k] * (tk_[k][a] * nz + nv[a] * tz);
    }
    for (int a = 0; a < 3; ++a) {
      gpos[4 * j + a] += ybar[a] / h;
      gpos[4 * i + a] -= ybar[a] / h;
    }
  }
}

/* Rows are dealt to the threads in fixed chunks; each thread sums into its own
 * buffer and the buffers are added in thread order (deterministic for a given
 * thread count). */
void orc_stencil_grad(int64_t n, const double *P, const uint8_t *model, const int64_t *row_ptr,
                      const int32_t *col, const orc_params *prm, const double *fields,
                      const double *gout, double *gpos) {
  for (int64_t k = 0; k < 4 * n; ++k) gpos[k] = 0.0;
  if (n <= 0) return;
  int nth = 1;
#ifdef _OPENMP
  nth = omp_get_max_threads();
#endif
  double *buf = (double *)calloc((size_t)nth * (size_t)(4 * n), sizeof(double));
  if (!buf) return;
#pragma omp parallel num_threads(nth)
  {
    int t = 0;
#ifdef _OPENMP
    t = omp_get_thread_num();
#endif
    double *g = buf + (size_t)t * (size_t)(4 * n);
#pragma omp for schedule(static, 64)
    for (int64_t i = 0; i < n; ++i) {
      /* a row whose 16 output gradients are all zero contributes exactly zero
         (every term of its adjoint is a product with gbar = 0): skip it */
      int live = 0;
      for (int k = 0; k < 16; ++k) live |= gout[16 * i + k] != 0.0;
      if (!live) continue;
      stencil_grad_one(i, P, model, row_ptr, col, prm, fields, gout, g);
    }
  }
#pragma omp parallel for schedule(static)
  for (int64_t k = 0; k < 4 * n; ++k) {
    double s = 0.0;
    for (int t = 0; t < nth; ++t) s += buf[(size_t)t * (size_t)(4 * n) + k];
    gpos[k] = s;
  }
  free(buf);
}

/* Eq. GFDM_Definition: d*_i u = sum_{j in S_i} c*_ij u_j, for the four fields. */
void orc_apply(int64_t n, const int64_t *row_ptr, const int32_t *col, const double *coef,
               const double *fields, const int64_t *rows, int64_t nrows, double *out) {
  int64_t cnt = rows ? nrows : n;
#pragma omp parallel for schedule(dynamic, 256)
  for (int64_t r = 0; r < cnt; ++r) {
    int64_t i = rows ? rows[r] : r;
    double acc[4][4] = {{0}};
    for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
      int64_t j = col[e];
      for (int f = 0; f < 4; ++f)
        for (int op = 0; op < 4; ++op) acc[f][op] += coef[4 * e + op] * fields[4 * j + f];
    }
    for (int f = 0; f < 4; ++f)
      for (int op = 0; op < 4; ++op) out[16 * i + 4 * f + op] = acc[f][op];
  }
}

void orc_apply_T(int64_t n, const int64_t *row_ptr, const int32_t *col, const double *coef,
                 const double *gout, double *gfields) {
  for (int64_t j = 0; j < 4 * n; ++j) gfields[j] = 0.0;
  for (int64_t i = 0; i < n; ++i)
    for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
      int64_t j = col[e];
      for (int f = 0; f < 4; ++f)
        for (int op = 0; op < 4; ++op)
          gfields[4 * j + f] += coef[4 * e + op] * gout[16 * i + 4 * f + op];
    }
}

/* ---------------------------------------------------------------------------
 * Model transition, Sec. 5.
 * ------------------------------------------------------------------------- */
static void copy_particle(const orc_state *in, int64_t i, orc_state *out, int64_t o) {
  for (int a = 0; a < 4; ++a) {
    out->pos_h[4 * o + a] = in->pos_h[4 * i + a];
    out->vp[4 * o + a] = in->vp[4 * i + a];
    out->normal[4 * o + a] = in->normal[4 * i + a];
  }
  out->rho[o] = in->rho[i];
  out->eta[o] = in->eta[i];
  out->mass[o] = in->mass[i];
  out->diam[o] = in->diam[i];
  out->hfilm[o] = in->hfilm[i];
  out->h3d[o] = in->h3d[i];
  out->model[o] = in->model[i];
  out->type[o] = in->type[i];
  out->last[o] = 0;
}

int64_t orc_remap(int64_t n, const orc_state *in, const uint8_t *flag, const int64_t *row_ptr,
                  const int32_t *col, const orc_params *prm, orc_state *out, int64_t cap_out,
                  int32_t *old2new) {
  const double *P = in->pos_h;
  /* Alg. 3, first loop: interior / free-surface 3D neighbours of particles
   * flagged 3D -> 2D become deletion candidates.  Second loop: each candidate
   * b finds its nearest 3D wall particle j^w in S_b (ties: lower index); it is
   * mapped onto j^w (b in T_{j^w}) when j^w is flagged, otherwise kept. */
  int32_t *owner = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
  for (int64_t b = 0; b < n; ++b) {
    owner[b] = -1;
    if (in->model[b] != M3D || in->type[b] == T_WALL) continue;
    int cand = 0;
    for (int64_t e = row_ptr[b]; e < row_ptr[b + 1]; ++e) {
      int64_t j = col[e];
      if (in->model[j] == M3D && flag[j] == 1) cand = 1;
    }
    if (!cand) continue;
    int64_t jw = -1;
    double best = INFINITY;
    for (int64_t e = row_ptr[b]; e < row_ptr[b + 1]; ++e) {
      int64_t j = col[e];
      if (in->model[j] != M3D || in->type[j] != T_WALL) continue;
      double d2 = dist2(P, b, j);
      if (d2 < best || (d2 == best && j < jw)) {
        best = d2;
        jw = j;
      }
    }
    if (jw >= 0 && flag[jw] == 1) owner[b] = (int32_t)jw;
  }
  /* Alg. 4: number of particles added along the normal of each 2D particle
   * flagged 2D -> 3D: gamma = ceil(H / psi~), psi~ = (r_min + r_max) h / 2. */
  int64_t n_keep = 0, n_new = 0;
  for (int64_t i = 0; i < n; ++i) {
    if (owner[i] < 0) ++n_keep;
    if (flag[i] == 2 && in->model[i] == M2D) {
      double psi_t = prm->c_psi * in->h3d[i];
      double H = in->hfilm[i];
      n_new += H > 0.0 ? (int64_t)ceil(H / psi_t) : 0;
    }
  }
  int64_t n_out = n_keep + n_new;
  if (n_out > cap_out) {
    free(owner);
    return -n_out;
  }
  int64_t o = 0;
  for (int64_t i = 0; i < n; ++i) {
    if (owner[i] >= 0) {
      old2new[i] = -1;
      continue;
    }
    old2new[i] = (int32_t)o;
    copy_particle(in, i, out, o);
    if (flag[i] == 1 && in->model[i] == M3D) {
      /* 3D -> 2D data mapping (Sec. 5.1): average v, p, rho, eta over {i} u T_i,
       * lump mass, droplet diameter from m = rho V, film height = largest
       * normal distance to T_i. */
      double vp[4], rho = in->rho[i], eta = in->eta[i], m = in->mass[i], H = 0.0;
      int64_t cnt = 0;
      for (int a = 0; a < 4; ++a) vp[a] = in->vp[4 * i + a];
      for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
        int64_t b = col[e];
        if (owner[b] != i) continue;
        for (int a = 0; a < 4; ++a) vp[a] += in->vp[4 * b + a];
        rho += in->rho[b];
        eta += in->eta[b];
        m += in->mass[b];
        double dn = fabs((P[4 * b] - P[4 * i]) * in->normal[4 * i] +
                         (P[4 * b + 1] - P[4 * i + 1]) * in->normal[4 * i + 1] +
                         (P[4 * b + 2] - P[4 * i + 2]) * in->normal[4 * i + 2]);
        if (dn > H) H = dn;
        ++cnt;
      }
      double k = 1.0 + (double)cnt;
      for (int a = 0; a < 4; ++a) out->vp[4 * o + a] = vp[a] / k;
      out->rho[o] = rho / k;
      out->eta[o] = eta / k;
      out->mass[o] = m;
      out->diam[o] = cbrt(6.0 * m / (M_PI * out->rho[o]));
      out->hfilm[o] = H;
      out->model[o] = M2D;
      out->type[o] = T_WALL;
      out->last[o] = 1;
    } else if (flag[i] == 2 && in->model[i] == M2D) {
      double psi_t = prm->c_psi * in->h3d[i];
      double H = in->hfilm[i];
      int64_t g = H > 0.0 ? (int64_t)ceil(H / psi_t) : 0;
      double m = in->mass[i] / (1.0 + (double)g);
      out->mass[o] = m;
      out->diam[o] = cbrt(6.0 * m / (M_PI * in->rho[i]));
      out->pos_h[4 * o + 3] = in->h3d[i];
      out->hfilm[o] = 0.0;
      out->model[o] = M3D;
      out->type[o] = T_WALL;
      out->last[o] = 1;
    }
    ++o;
  }
  /* Alg. 4, particle addition: x_i + k psi n_i, k = 1..gamma, psi = H/gamma,
   * the farthest one free surface; v, p, rho, eta copied; m_i/(1+gamma) each. */
  for (int64_t i = 0; i < n; ++i) {
    if (!(flag[i] == 2 && in->model[i] == M2D)) continue;
    double psi_t = prm->c_psi * in->h3d[i];
    double H = in->hfilm[i];
    int64_t g = H > 0.0 ? (int64_t)ceil(H / psi_t) : 0;
    if (g == 0) continue;
    double psi = H / (double)g;
    double m = in->mass[i] / (1.0 + (double)g);
    for (int64_t k = 1; k <= g; ++k) {
      copy_particle(in, i, out, o);
      double kp = (double)k * psi;
      for (int a = 0; a < 3; ++a) out->pos_h[4 * o + a] = P[4 * i + a] + kp * in->normal[4 * i + a];
      out->pos_h[4 * o + 3] = in->h3d[i];
      out->mass[o] = m;
      out->diam[o] = cbrt(6.0 * m / (M_PI * in->rho[i]));
      out->hfilm[o] = 0.0;
      out->model[o] = M3D;
      out->type[o] = (k == g) ? T_FS : T_INT;
      out->last[o] = 1;
      ++o;
    }
  }
  free(owner);
  return n_out;
}

/* ---------------------------------------------------------------------------
 * Buffer zone, Sec. 5.3 (Alg. 5), first loop: a particle is a ghost source
 * when a particle of the other model lies in its neighbourhood S_i.
 * ------------------------------------------------------------------------- */
void orc_ghost_sources(int64_t n, const uint8_t *model, const int64_t *row_ptr,
                       const int32_t *col, uint8_t *src) {
  for (int64_t i = 0; i < n; ++i) {
    src[i] = 0;
    for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e)
      if (model[col[e]] != model[i]) src[i] = 1;
  }
}
