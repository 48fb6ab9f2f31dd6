// stencil_common.cuh -- device pieces shared by the GFDM stencil build and its
// adjoint: monomial bases, the least-squares weight, packed Cholesky and solves.
#pragma once
#include <math.h>

#include "internal.cuh"

namespace mafp {

constexpr int kStThreads = 128;

template <int M> struct Basis;
template <> struct Basis<10> {
  static constexpr int NA = 55;   // packed lower triangle of A
  static constexpr int NR = 4;    // right-hand sides: d/dx, d/dy, d/dz, Laplacian
};
template <> struct Basis<6> {
  static constexpr int NA = 21;
  static constexpr int NR = 3;    // d/dxi, d/deta, surface Laplacian
};

__host__ __device__ constexpr int pad_to(int v, int g) { return ((v + g - 1) / g) * g; }
__host__ __device__ constexpr int pk(int r, int c) { return r * (r + 1) / 2 + c; }

// Distinct moments of the basis products.  Every entry A_rc = sum_j w_j p_r p_c
// is the weighted moment of the monomial p_r p_c (degree <= 4); equal
// monomials give equal entries, so only the distinct ones are summed: 35 of
// the 55 entries in 3D, 15 of the 21 in 2D.  Moment m is accumulated as
// (w p_rep_r[m]) p_rep_c[m]; entry pk(r, c) reads moment idx[pk(r, c)].
template <int M>
struct MomentTable {
  int n = 0;
  int rep_r[Basis<M>::NA] = {};
  int rep_c[Basis<M>::NA] = {};
  int idx[Basis<M>::NA] = {};
};
// Exponents of the basis monomials: (1, qx, qy, qz, qx^2, qy^2, qz^2, qx qy,
// qx qz, qy qz) in 3D, (1, xi, eta, xi^2, xi eta, eta^2) in 2D.
template <int M>
constexpr MomentTable<M> make_moment_table() {
  int e[10][3] = {{0, 0, 0}, {1, 0, 0}, {0, 1, 0}, {0, 0, 1}, {2, 0, 0},
                  {0, 2, 0}, {0, 0, 2}, {1, 1, 0}, {1, 0, 1}, {0, 1, 1}};
  if (M == 6) {
    const int e2[6][3] = {{0, 0, 0}, {1, 0, 0}, {0, 1, 0}, {2, 0, 0}, {1, 1, 0}, {0, 2, 0}};
    for (int r = 0; r < 6; ++r)
      for (int a = 0; a < 3; ++a) e[r][a] = e2[r][a];
  }
  MomentTable<M> t;
  int sum[Basis<M>::NA][3] = {};
  for (int r = 0; r < M; ++r)
    for (int c = 0; c <= r; ++c) {
      const int s0 = e[r][0] + e[c][0], s1 = e[r][1] + e[c][1], s2 = e[r][2] + e[c][2];
      int m = 0;
      while (m < t.n && !(sum[m][0] == s0 && sum[m][1] == s1 && sum[m][2] == s2)) ++m;
      if (m == t.n) {
        sum[m][0] = s0;
        sum[m][1] = s1;
        sum[m][2] = s2;
        t.rep_r[m] = r;
        t.rep_c[m] = c;
        ++t.n;
      }
      t.idx[r * (r + 1) / 2 + c] = m;
    }
  return t;
}
template <int M>
struct Moments {
  static constexpr MomentTable<M> T = make_moment_table<M>();
  static constexpr int N = T.n;
};
static_assert(Moments<10>::N == 35 && Moments<6>::N == 15, "distinct moments of degree <= 4");

// Every entry (r, c) reads a moment whose representative pair multiplies to the
// same monomial, and distinct moments are distinct monomials (checked while
// compiling, from the exponents written out again here).
template <int M>
constexpr bool moment_table_consistent() {
  int e[10][3] = {{0, 0, 0}, {1, 0, 0}, {0, 1, 0}, {0, 0, 1}, {2, 0, 0},
                  {0, 2, 0}, {0, 0, 2}, {1, 1, 0}, {1, 0, 1}, {0, 1, 1}};
  if (M == 6) {
    const int e2[6][3] = {{0, 0, 0}, {1, 0, 0}, {0, 1, 0}, {2, 0, 0}, {1, 1, 0}, {0, 2, 0}};
    for (int r = 0; r < 6; ++r)
      for (int a = 0; a < 3; ++a) e[r][a] = e2[r][a];
  }
  constexpr MomentTable<M> T = make_moment_table<M>();
  for (int r = 0; r < M; ++r)
    for (int c = 0; c <= r; ++c) {
      const int m = T.idx[r * (r + 1) / 2 + c];
      if (m < 0 || m >= T.n) return false;
      for (int a = 0; a < 3; ++a)
        if (e[r][a] + e[c][a] != e[T.rep_r[m]][a] + e[T.rep_c[m]][a]) return false;
    }
  for (int m = 0; m < T.n; ++m)
    for (int k = 0; k < m; ++k) {
      bool same = true;
      for (int a = 0; a < 3; ++a)
        same = same && (e[T.rep_r[m]][a] + e[T.rep_c[m]][a] == e[T.rep_r[k]][a] + e[T.rep_c[k]][a]);
      if (same) return false;
    }
  return true;
}
static_assert(moment_table_consistent<10>() && moment_table_consistent<6>(),
              "moment table: entries and representatives disagree");

// Add w p p^T of one neighbour to the distinct moments.
template <int M, typename C, int VM>
__device__ __forceinline__ void add_moments(C (&mom)[VM], C w, const C (&p)[M]) {
  constexpr MomentTable<M> T = Moments<M>::T;
#pragma unroll
  for (int m = 0; m < Moments<M>::N; ++m) mom[m] += (w * p[T.rep_r[m]]) * p[T.rep_c[m]];
}

template <typename C>
struct StParams {
  C alpha, ea, inv_den;   // W(s) = (exp(-alpha s^2) - ea) * inv_den, s <= 1
  C piv_tol_rel;          // pivot <= tol * trace -> rank deficient (FP64) / fall back (FP32)
  C cond_max;
};

template <typename C>
__device__ __forceinline__ C weight_w(C s2, const StParams<C> &sp) {
  return s2 <= C(1) ? (exp(-sp.alpha * s2) - sp.ea) * sp.inv_den : C(0);
}

// Monomial basis at one neighbour; returns w (0 for j outside the unit support).
// With e_out, also exp(-alpha s^2) (for W'), from the same exponential as w.
template <int M, typename C, typename V>
__device__ __forceinline__ C basis_at(const V &xi, const V &xj, C hinv, const C (&t1)[3],
                                      const C (&t2)[3], const StParams<C> &sp, C (&p)[M],
                                      C *e_out = nullptr) {
  const C dx = C(xj.x) - C(xi.x), dy = C(xj.y) - C(xi.y), dz = C(xj.z) - C(xi.z);
  const C s2 = ((dx * dx + dy * dy) + dz * dz) * (hinv * hinv);
  C w;
  if (e_out) {
    const C e = exp(-sp.alpha * s2);
    *e_out = e;
    w = s2 <= C(1) ? (e - sp.ea) * sp.inv_den : C(0);
  } else {
    w = weight_w<C>(s2, sp);
  }
  if constexpr (M == 10) {
    const C qx = dx * hinv, qy = dy * hinv, qz = dz * hinv;
    p[0] = C(1); p[1] = qx; p[2] = qy; p[3] = qz;
    p[4] = qx * qx; p[5] = qy * qy; p[6] = qz * qz;
    p[7] = qx * qy; p[8] = qx * qz; p[9] = qy * qz;
  } else {
    const C xi_ = (dx * t1[0] + dy * t1[1] + dz * t1[2]) * hinv;
    const C et_ = (dx * t2[0] + dy * t2[1] + dz * t2[2]) * hinv;
    p[0] = C(1); p[1] = xi_; p[2] = et_;
    p[3] = xi_ * xi_; p[4] = xi_ * et_; p[5] = et_ * et_;
  }
  return w;
}

// The same monomials rebuilt from a cached (q, w): q = (x_j - x_i) / h_i in 3D,
// (xi, eta) in 2D, with the products taken exactly as basis_at takes them.
template <int M, typename C>
__device__ __forceinline__ void basis_from_q(const float4 &c, C (&p)[M]) {
  if constexpr (M == 10) {
    const C qx = c.x, qy = c.y, qz = c.z;
    p[0] = C(1); p[1] = qx; p[2] = qy; p[3] = qz;
    p[4] = qx * qx; p[5] = qy * qy; p[6] = qz * qz;
    p[7] = qx * qy; p[8] = qx * qz; p[9] = qy * qz;
  } else {
    const C xi_ = c.x, et_ = c.y;
    p[0] = C(1); p[1] = xi_; p[2] = et_;
    p[3] = xi_ * xi_; p[4] = xi_ * et_; p[5] = et_ * et_;
  }
}

// Right-hand side k (unscaled: the 1/h and 1/h^2 factors are applied to the output).
template <int M, typename C>
__device__ __forceinline__ C rhs(int k, int r) {
  if constexpr (M == 10) {
    if (k < 3) return r == k + 1 ? C(1) : C(0);
    return (r >= 4 && r <= 6) ? C(2) : C(0);
  } else {
    if (k < 2) return r == k + 1 ? C(1) : C(0);
    return (r == 3 || r == 5) ? C(2) : C(0);
  }
}

// In-register Cholesky of the packed matrix L (lower), returns false when a
// pivot is <= tol.  invd gets 1/L_kk; pmin / pmax the extreme pivots.
template <int M, typename C>
__device__ __forceinline__ bool cholesky(C (&L)[Basis<M>::NA], C (&invd)[M], C tol, C &pmin,
                                         C &pmax) {
  pmin = C(INFINITY);
  pmax = C(0);
  bool ok = true;
#pragma unroll
  for (int k = 0; k < M; ++k) {
    C d = L[pk(k, k)];
#pragma unroll
    for (int l = 0; l < k; ++l) d -= L[pk(k, l)] * L[pk(k, l)];
    ok = ok && (d > tol);
    const C lkk = sqrt(d > tol ? d : C(1));
    L[pk(k, k)] = lkk;
    invd[k] = C(1) / lkk;
    pmin = lkk < pmin ? lkk : pmin;
    pmax = lkk > pmax ? lkk : pmax;
#pragma unroll
    for (int r = k + 1; r < M; ++r) {
      C s = L[pk(r, k)];
#pragma unroll
      for (int l = 0; l < k; ++l) s -= L[pk(r, l)] * L[pk(k, l)];
      L[pk(r, k)] = s * invd[k];
    }
  }
  return ok;
}

template <int M, typename C>
__device__ __forceinline__ void chol_solve(const C (&L)[Basis<M>::NA], const C (&invd)[M],
                                           const C (&b)[M], C (&x)[M]) {
  C y[M];
#pragma unroll
  for (int r = 0; r < M; ++r) {
    C s = b[r];
#pragma unroll
    for (int l = 0; l < r; ++l) s -= L[pk(r, l)] * y[l];
    y[r] = s * invd[r];
  }
#pragma unroll
  for (int r = M - 1; r >= 0; --r) {
    C s = y[r];
#pragma unroll
    for (int l = r + 1; l < M; ++l) s -= L[pk(l, r)] * x[l];
    x[r] = s * invd[r];
  }
}

// Same solve with the factor read from shared memory (every lane of the group
// reads the same address: a broadcast), which keeps the 55 entries of L out
// of the registers during the refinement pass.
template <int M, typename C>
__device__ __forceinline__ void chol_solve_s(const C *L, const C (&invd)[M], const C (&b)[M],
                                             C (&x)[M]) {
  C y[M];
#pragma unroll
  for (int r = 0; r < M; ++r) {
    C s = b[r];
#pragma unroll
    for (int l = 0; l < r; ++l) s -= L[pk(r, l)] * y[l];
    y[r] = s * invd[r];
  }
#pragma unroll
  for (int r = M - 1; r >= 0; --r) {
    C s = y[r];
#pragma unroll
    for (int l = r + 1; l < M; ++l) s -= L[pk(l, r)] * x[l];
    x[r] = s * invd[r];
  }
}

// U neighbours of one lane (entries e0, e0 + G, ..., e0 + (U-1) G of the row),
// gathered before any of them is used so that their loads are in flight
// together.  Slots past the row end load particle i itself and are marked
// invalid, as are neighbours of the other model.
template <int U, int G, typename V>
__device__ __forceinline__ void gather_row(long long e0, long long e1, int64_t i, uint8_t mi,
                                           const int32_t *col, const V *pos,
                                           const uint8_t *model, V (&x)[U], bool (&ok)[U]) {
  int j[U];
#pragma unroll
  for (int u = 0; u < U; ++u) {
    const long long e = e0 + (long long)u * G;
    j[u] = e < e1 ? col[e] : (int)i;
  }
  uint8_t m[U];
#pragma unroll
  for (int u = 0; u < U; ++u) {
    x[u] = ld4(pos + j[u]);
    m[u] = model[j[u]];
  }
#pragma unroll
  for (int u = 0; u < U; ++u) ok[u] = (e0 + (long long)u * G < e1) && m[u] == mi;
}

// The same, also gathering a per-particle field record of every neighbour.
template <int U, int G, typename V>
__device__ __forceinline__ void gather_row_f(long long e0, long long e1, int64_t i, uint8_t mi,
                                             const int32_t *col, const V *pos,
                                             const uint8_t *model, const V *fld, V (&x)[U],
                                             V (&f)[U], int (&j)[U], bool (&ok)[U]) {
#pragma unroll
  for (int u = 0; u < U; ++u) {
    const long long e = e0 + (long long)u * G;
    j[u] = e < e1 ? col[e] : (int)i;
  }
  uint8_t m[U];
#pragma unroll
  for (int u = 0; u < U; ++u) {
    x[u] = ld4(pos + j[u]);
    f[u] = ld4(fld + j[u]);
    m[u] = model[j[u]];
  }
#pragma unroll
  for (int u = 0; u < U; ++u) ok[u] = (e0 + (long long)u * G < e1) && m[u] == mi;
}

// ---- software-pipelined row walk (FP32 storage) ---------------------------
// A lane walks its entries e = b + lane + k G (k = 0, 1, ...) of row i.  The
// neighbour records (position, and with FIELDS its field record) are copied by
// cp.async into a ring of D slots in shared memory D entries before they are
// used; the column index is loaded 2D entries before and the neighbour's model
// byte D entries before (registers).  The dependent loads col -> pos / fields
// then overlap the arithmetic of the entries in between instead of stalling at
// every entry, and the records in flight hold no registers.
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;\n" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// Slots of the block's ring: record r of slot s of thread t sits at
// ((s * R + r) * kStThreads + t), so a warp's lanes touch consecutive 16-byte
// words (no bank conflicts).  body(xj, fj, j, ok) runs once per entry of the
// lane in row order; ok = the entry exists and j has the model of i (fj is xj
// when !FIELDS; for !ok both may hold stale data and must not be used).
template <int D, int G, bool FIELDS, typename F>
__device__ __forceinline__ void stream_row(long long b, long long e1, uint8_t mi,
                                           const int32_t *col, const float4 *pos,
                                           const uint8_t *model, const float4 *fld,
                                           float4 *ring, F &&body) {
  constexpr int R = FIELDS ? 2 : 1;
  const int t = threadIdx.x;
  const int lane = t & (G - 1);
  const int nloc = e1 > b + lane ? (int)((e1 - b - lane + G - 1) / G) : 0;
  auto colk = [&](int k) -> int {
    const long long e = b + lane + (long long)k * G;
    return e < e1 ? col[e] : -1;
  };
  auto slot = [&](int s, int r) -> float4 * { return ring + (s * R + r) * kStThreads + t; };
  int js[D], jn[D];
  unsigned ms[D];
#pragma unroll
  for (int s = 0; s < D; ++s) js[s] = colk(s);
#pragma unroll
  for (int s = 0; s < D; ++s) {
    ms[s] = 0xffu;
    if (js[s] >= 0) {
      ms[s] = model[js[s]];
      cp_async16(slot(s, 0), pos + js[s]);
      if constexpr (FIELDS) cp_async16(slot(s, 1), fld + js[s]);
    }
    cp_async_commit();
  }
#pragma unroll
  for (int s = 0; s < D; ++s) jn[s] = colk(D + s);
  for (int k0 = 0; k0 < nloc; k0 += D) {
#pragma unroll
    for (int s = 0; s < D; ++s) {
      cp_async_wait<D - 1>();   // the oldest group: this slot's records
      const float4 xj = *slot(s, 0);
      float4 fj = xj;
      if constexpr (FIELDS) fj = *slot(s, 1);
      const int j = js[s];
      body(xj, fj, j, j >= 0 && ms[s] == (unsigned)mi);
      // refill the slot (its records are consumed) with the entry D further on
      const int jx = jn[s];
      js[s] = jx;
      ms[s] = 0xffu;
      if (jx >= 0) {
        ms[s] = model[jx];
        cp_async16(slot(s, 0), pos + jx);
        if constexpr (FIELDS) cp_async16(slot(s, 1), fld + jx);
      }
      cp_async_commit();
      jn[s] = colk(k0 + s + 2 * D);
    }
  }
  cp_async_wait<0>();
}

template <int M, int G>
struct StSmem {
  static constexpr int NA = Basis<M>::NA, NR = Basis<M>::NR;
  static constexpr int SCR = pad_to(NA, G) > pad_to(NR * M, G) ? pad_to(NA, G) : pad_to(NR * M, G);
  static constexpr int PER_GROUP = SCR + NA;   // reduce scratch + Cholesky factor
};


template <typename C>
inline StParams<C> make_params(const mafp_params &p, double piv_tol) {
  StParams<C> sp;
  const double ea = exp(-p.alpha_w);
  sp.alpha = (C)p.alpha_w;
  sp.ea = (C)ea;
  sp.inv_den = (C)(1.0 / (1.0 - ea));
  sp.piv_tol_rel = (C)piv_tol;
  sp.cond_max = (C)p.cond_fp64;
  return sp;
}

}  // namespace mafp
