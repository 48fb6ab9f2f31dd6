// classify.cu -- model-transition detection of Sec. 4 (Alg. 2, Eq. Height,
// Eq. 2Dto3Dcond) and the smoothing of Sec. 4.3.  One warp per particle; lanes
// stride over the neighbour row and reduce with shuffles.  The FP32 path takes
// every decision that lies within a band of its threshold again in FP64.
#include <climits>

#include "internal.cuh"

namespace mafp {

constexpr int kClsThreads = 128;

// ------------------------------------------------------------ FP64 Jacobi
// Cyclic Jacobi for a symmetric 3x3 matrix a = (xx, yy, zz, xy, xz, yz):
// lam descending, W[k] = unit eigenvector of lam[k].
__device__ void eig3_jacobi(const double a6[6], double lam[3], double W[3][3]) {
  double A[3][3] = {{a6[0], a6[3], a6[4]}, {a6[3], a6[1], a6[5]}, {a6[4], a6[5], a6[2]}};
  double V[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
  double tot = 0.0;
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) tot += A[r][c] * A[r][c];
  for (int sweep = 0; sweep < 50; ++sweep) {
    double off = A[0][1] * A[0][1] + A[0][2] * A[0][2] + A[1][2] * A[1][2];
    if (off == 0.0 || off <= 1e-40 * tot) break;
    for (int pq = 0; pq < 3; ++pq) {
      const int p = pq == 2 ? 1 : 0, q = pq == 0 ? 1 : 2;
      const double apq = A[p][q];
      if (apq == 0.0) continue;
      const double tau = (A[q][q] - A[p][p]) / (2.0 * apq);
      const double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
      const double c = 1.0 / sqrt(1.0 + t * t), s = t * c;
      // A <- J^T A J with J = identity except J_pp = J_qq = c, J_pq = s, J_qp = -s
      for (int k = 0; k < 3; ++k) {
        const double akp = A[k][p], akq = A[k][q];
        A[k][p] = c * akp - s * akq;
        A[k][q] = s * akp + c * akq;
      }
      for (int k = 0; k < 3; ++k) {
        const double apk = A[p][k], aqk = A[q][k];
        A[p][k] = c * apk - s * aqk;
        A[q][k] = s * apk + c * aqk;
      }
      A[p][q] = A[q][p] = 0.0;
      for (int k = 0; k < 3; ++k) {
        const double vkp = V[k][p], vkq = V[k][q];
        V[k][p] = c * vkp - s * vkq;
        V[k][q] = s * vkp + c * vkq;
      }
    }
  }
  int o[3] = {0, 1, 2};
  for (int a = 0; a < 3; ++a)
    for (int b = a + 1; b < 3; ++b)
      if (A[o[b]][o[b]] > A[o[a]][o[a]]) {
        int t = o[a]; o[a] = o[b]; o[b] = t;
      }
  for (int k = 0; k < 3; ++k) {
    lam[k] = A[o[k]][o[k]];
    for (int r = 0; r < 3; ++r) W[k][r] = V[r][o[k]];
  }
}

// ------------------------------------------------------- FP32 closed form
// Eigenvalues from the trigonometric solution of the characteristic
// polynomial of the shifted, scaled matrix; the eigenvector of the better
// separated extreme eigenvalue from the largest cross product of two rows of
// (B - lambda I); the other two from the 2x2 problem on its orthogonal
// complement; eigenvalues refined as Rayleigh quotients.
__device__ __forceinline__ void cross3(const float a[3], const float b[3], float c[3]) {
  c[0] = a[1] * b[2] - a[2] * b[1];
  c[1] = a[2] * b[0] - a[0] * b[2];
  c[2] = a[0] * b[1] - a[1] * b[0];
}
__device__ __forceinline__ float dot3(const float a[3], const float b[3]) {
  return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}
__device__ __forceinline__ void matvec6(const float b[6], const float v[3], float o[3]) {
  o[0] = b[0] * v[0] + b[3] * v[1] + b[4] * v[2];
  o[1] = b[3] * v[0] + b[1] * v[1] + b[5] * v[2];
  o[2] = b[4] * v[0] + b[5] * v[1] + b[2] * v[2];
}

__device__ void null_vector(const float b[6], float l, float v[3]) {
  const float r0[3] = {b[0] - l, b[3], b[4]};
  const float r1[3] = {b[3], b[1] - l, b[5]};
  const float r2[3] = {b[4], b[5], b[2] - l};
  float c0[3], c1[3], c2[3];
  cross3(r0, r1, c0);
  cross3(r0, r2, c1);
  cross3(r1, r2, c2);
  const float n0 = dot3(c0, c0), n1 = dot3(c1, c1), n2 = dot3(c2, c2);
  const float *c = c0;
  float nn = n0;
  if (n1 > nn) { c = c1; nn = n1; }
  if (n2 > nn) { c = c2; nn = n2; }
  if (nn > 0.0f) {
    const float inv = rsqrtf(nn);
    v[0] = c[0] * inv; v[1] = c[1] * inv; v[2] = c[2] * inv;
  } else {
    v[0] = 1.0f; v[1] = 0.0f; v[2] = 0.0f;
  }
}

__device__ void eig3_closed(const float a6[6], float lam[3], float W[3][3], float *gap_rel) {
  float s = 0.0f;
  for (int k = 0; k < 6; ++k) s = fmaxf(s, fabsf(a6[k]));
  if (!(s > 0.0f)) {
    for (int k = 0; k < 3; ++k) {
      lam[k] = 0.0f;
      for (int r = 0; r < 3; ++r) W[k][r] = k == r ? 1.0f : 0.0f;
    }
    *gap_rel = 0.0f;
    return;
  }
  const float is = 1.0f / s;
  float b[6];
  for (int k = 0; k < 6; ++k) b[k] = a6[k] * is;
  const float q = (b[0] + b[1] + b[2]) * (1.0f / 3.0f);
  const float c0 = b[0] - q, c1 = b[1] - q, c2 = b[2] - q;
  const float p2 = (c0 * c0 + c1 * c1 + c2 * c2 + 2.0f * (b[3] * b[3] + b[4] * b[4] + b[5] * b[5])) *
                   (1.0f / 6.0f);
  const float p = sqrtf(p2);
  float l1, l2, l3;
  float w1[3], w2[3], w3[3];
  if (p < 1e-12f) {
    l1 = l2 = l3 = q;
    w1[0] = 1; w1[1] = 0; w1[2] = 0;
    w2[0] = 0; w2[1] = 1; w2[2] = 0;
    w3[0] = 0; w3[1] = 0; w3[2] = 1;
  } else {
    const float det = c0 * (c1 * c2 - b[5] * b[5]) - b[3] * (b[3] * c2 - b[5] * b[4]) +
                      b[4] * (b[3] * b[5] - c1 * b[4]);
    float r = det / (2.0f * p2 * p);
    r = fminf(1.0f, fmaxf(-1.0f, r));
    const float phi = acosf(r) * (1.0f / 3.0f);
    l1 = q + 2.0f * p * cosf(phi);
    l3 = q + 2.0f * p * cosf(phi + 2.0943951023931957f);
    l2 = 3.0f * q - l1 - l3;
    float u[3];
    const bool top = (l1 - l2) >= (l2 - l3);
    null_vector(b, top ? l1 : l3, u);
    // orthonormal basis (e, f) of the complement of u
    float ax[3] = {0, 0, 0};
    const float au0 = fabsf(u[0]), au1 = fabsf(u[1]), au2 = fabsf(u[2]);
    ax[(au0 <= au1 && au0 <= au2) ? 0 : (au1 <= au2 ? 1 : 2)] = 1.0f;
    float e[3], f[3];
    cross3(u, ax, e);
    const float ie = rsqrtf(dot3(e, e));
    e[0] *= ie; e[1] *= ie; e[2] *= ie;
    cross3(u, e, f);
    float Be[3], Bf[3];
    matvec6(b, e, Be);
    matvec6(b, f, Bf);
    const float m00 = dot3(e, Be), m01 = dot3(e, Bf), m11 = dot3(f, Bf);
    const float th = 0.5f * atan2f(2.0f * m01, m00 - m11);
    const float ct = cosf(th), st = sinf(th);
    float ga[3], gb[3];  // ga: larger eigenvalue of the 2x2 block, gb: smaller
    for (int k = 0; k < 3; ++k) {
      ga[k] = ct * e[k] + st * f[k];
      gb[k] = -st * e[k] + ct * f[k];
    }
    if (top) {
      for (int k = 0; k < 3; ++k) { w1[k] = u[k]; w2[k] = ga[k]; w3[k] = gb[k]; }
    } else {
      for (int k = 0; k < 3; ++k) { w1[k] = ga[k]; w2[k] = gb[k]; w3[k] = u[k]; }
    }
  }
  // Rayleigh quotients on the scaled matrix, then undo the scaling
  float Bw[3];
  matvec6(b, w1, Bw); l1 = dot3(w1, Bw);
  matvec6(b, w2, Bw); l2 = dot3(w2, Bw);
  matvec6(b, w3, Bw); l3 = dot3(w3, Bw);
  // keep descending order (Rayleigh quotients may swap nearly equal values)
  if (l2 > l1) { float t = l1; l1 = l2; l2 = t; for (int k = 0; k < 3; ++k) { float x = w1[k]; w1[k] = w2[k]; w2[k] = x; } }
  if (l3 > l2) { float t = l2; l2 = l3; l3 = t; for (int k = 0; k < 3; ++k) { float x = w2[k]; w2[k] = w3[k]; w3[k] = x; } }
  if (l2 > l1) { float t = l1; l1 = l2; l2 = t; for (int k = 0; k < 3; ++k) { float x = w1[k]; w1[k] = w2[k]; w2[k] = x; } }
  lam[0] = l1 * s; lam[1] = l2 * s; lam[2] = l3 * s;
  for (int k = 0; k < 3; ++k) { W[0][k] = w1[k]; W[1][k] = w2[k]; W[2][k] = w3[k]; }
  *gap_rel = (l1 > 0.0f) ? (l2 - l3) / l1 : 0.0f;
}

// ------------------------------------------------------------ warp helpers
__device__ __forceinline__ float wsum(float v) { return group_sum<32>(v); }
__device__ __forceinline__ double wsum(double v) { return group_sum<32>(v); }

// Unweighted centroid and scatter matrix of the same-model part of S_i in
// coordinates (x - x_i)/h_i (Sec. 4.1.2), two passes, in type C.
template <typename C, typename V>
__device__ void covariance(int64_t i, const V *pos, const uint8_t *model, const long long *row_ptr,
                           const int32_t *col, C cov[6], int *m_out) {
  const int lane = threadIdx.x & 31;
  const V xi = ld4(pos + i);
  const uint8_t mi = model[i];
  const C hinv = C(1) / C(xi.w);
  const long long b = row_ptr[i], e1 = row_ptr[i + 1];
  C sx = 0, sy = 0, sz = 0;
  int m = 0;
  for (long long e = b + lane; e < e1; e += 32) {
    const int j = col[e];
    if (model[j] != mi) continue;
    const V xj = ld4(pos + j);
    sx += (C(xj.x) - C(xi.x)) * hinv;
    sy += (C(xj.y) - C(xi.y)) * hinv;
    sz += (C(xj.z) - C(xi.z)) * hinv;
    ++m;
  }
  m = group_sum<32>(m);
  sx = wsum(sx); sy = wsum(sy); sz = wsum(sz);
  const C inv_m = m > 0 ? C(1) / C(m) : C(0);
  const C cx = sx * inv_m, cy = sy * inv_m, cz = sz * inv_m;
  C a[6] = {0, 0, 0, 0, 0, 0};
  for (long long e = b + lane; e < e1; e += 32) {
    const int j = col[e];
    if (model[j] != mi) continue;
    const V xj = ld4(pos + j);
    const C dx = (C(xj.x) - C(xi.x)) * hinv - cx;
    const C dy = (C(xj.y) - C(xi.y)) * hinv - cy;
    const C dz = (C(xj.z) - C(xi.z)) * hinv - cz;
    a[0] += dx * dx; a[1] += dy * dy; a[2] += dz * dz;
    a[3] += dx * dy; a[4] += dx * dz; a[5] += dy * dz;
  }
#pragma unroll
  for (int k = 0; k < 6; ++k) cov[k] = wsum(a[k]);
  *m_out = m;
}

template <typename C, typename V, typename TV>
__device__ C film_height(int64_t i, const V *pos, const uint8_t *model, const TV *vol,
                         const long long *row_ptr, const int32_t *col, C alpha) {
  const int lane = threadIdx.x & 31;
  const V xi = ld4(pos + i);
  const long long b = row_ptr[i], e1 = row_ptr[i + 1];
  C H = 0;
  const C api = alpha / C(3.141592653589793);
  for (long long e = b + lane; e < e1; e += 32) {
    const int j = col[e];
    if (model[j] != MAFP_MODEL_2D) continue;
    const V xj = ld4(pos + j);
    const C dx = C(xj.x) - C(xi.x), dy = C(xj.y) - C(xi.y), dz = C(xj.z) - C(xi.z);
    const C d2 = (dx * dx + dy * dy) + dz * dz;
    const C hj = C(xj.w);
    const C ih2 = C(1) / (hj * hj);
    H += api * ih2 * exp(-alpha * d2 * ih2) * C(vol[j]);
  }
  return wsum(H);
}

template <typename T>
__global__ void __launch_bounds__(kClsThreads) k_classify(
    int64_t n, const vec4_t<T> *pos, const uint8_t *model, const uint8_t *type,
    const vec4_t<T> *normal, const T *vol, const T *h3d, const uint8_t *user,
    const long long *row_ptr, const int32_t *col, uint8_t *preflag, vec4_t<T> *eig,
    vec4_t<T> *frame, T *hfilm, uint8_t *near, mafp_params prm, DevStatus *st) {
  using V = vec4_t<T>;
  const int lane = threadIdx.x & 31;
  const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const double cth = cos(prm.theta_star);
  for (int64_t i = wid; i < n; i += nwarps) {
    const uint8_t mi = model[i], ti = type[i], ui = user[i];
    uint8_t pre = 0, nr = 0;
    T lam[3] = {0, 0, 0}, W[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}}, H = 0, eps = 0;
    bool did_pca = false, retake = false;
    if (mi == MAFP_MODEL_3D && ti == MAFP_TYPE_WALL) {
      // Sec. 4.1.1 resolution criterion over 3D neighbours j != i
      const long long b = row_ptr[i], e1 = row_ptr[i + 1];
      int fs = 0, in = 0;
      for (long long e = b + lane; e < e1; e += 32) {
        const int j = col[e];
        if (j == i || model[j] != MAFP_MODEL_3D) continue;
        const uint8_t tj = type[j];
        fs |= tj == MAFP_TYPE_FREE_SURFACE;
        in |= tj == MAFP_TYPE_INTERIOR;
      }
      fs = __any_sync(0xffffffffu, fs);
      in = __any_sync(0xffffffffu, in);
      did_pca = true;
      T cov[6];
      int m;
      covariance<T>(i, pos, model, row_ptr, col, cov, &m);
      T gap = 0;
      if constexpr (sizeof(T) == 4) {
        eig3_closed(cov, lam, W, &gap);
      } else {
        double l[3], w[3][3];
        eig3_jacobi(cov, l, w);
        for (int k = 0; k < 3; ++k) {
          lam[k] = l[k];
          for (int r = 0; r < 3; ++r) W[k][r] = w[k][r];
        }
      }
      eps = (lam[0] + lam[1]) > T(0) ? T(2) * lam[2] / (lam[0] + lam[1]) : T(INFINITY);
      if (fs) {
        const V nv = ld4(normal + i);
        T ndw = fabs(nv.x * W[2][0] + nv.y * W[2][1] + nv.z * W[2][2]);
        if constexpr (sizeof(T) == 4) {
          // retake in FP64 where the FP32 decision is not certain
          const bool eps_unsure = fabsf(eps - (float)prm.eps_lambda_max) <= (float)prm.eps_band;
          const bool eps_pass = eps < (float)prm.eps_lambda_max;
          const bool ang_unsure =
              fabsf(ndw - (float)cth) <= (float)prm.angle_band || gap < 1e-2f;
          if (eps_unsure || (eps_pass && ang_unsure)) {
            retake = true;
            double c64[6], l64[3], w64[3][3];
            int m64;
            covariance<double>(i, pos, model, row_ptr, col, c64, &m64);
            eig3_jacobi(c64, l64, w64);
            const double e64 = (l64[0] + l64[1]) > 0.0 ? 2.0 * l64[2] / (l64[0] + l64[1]) : INFINITY;
            const double d64 = fabs((double)nv.x * w64[2][0] + (double)nv.y * w64[2][1] +
                                    (double)nv.z * w64[2][2]);
            const bool pass = (e64 < prm.eps_lambda_max) && (d64 >= cth);
            pre = (pass || (ui & MAFP_USER_TO_2D)) ? 1 : 0;
            if (!(ui & MAFP_USER_TO_2D)) {
              const bool en = fabs(e64 - prm.eps_lambda_max) <= prm.near_rel * prm.eps_lambda_max;
              const bool an = fabs(d64 - cth) <= prm.near_rel;
              if ((en && d64 >= cth) || (an && e64 < prm.eps_lambda_max) || (en && an)) nr = 1;
            }
            for (int k = 0; k < 3; ++k) {
              lam[k] = (T)l64[k];
              for (int r = 0; r < 3; ++r) W[k][r] = (T)w64[k][r];
            }
            eps = (T)e64;
          } else {
            const bool pass = eps_pass && (ndw >= (float)cth);
            pre = (pass || (ui & MAFP_USER_TO_2D)) ? 1 : 0;
          }
        } else {
          const bool pass = (eps < prm.eps_lambda_max) && (ndw >= cth);
          pre = (pass || (ui & MAFP_USER_TO_2D)) ? 1 : 0;
          if (!(ui & MAFP_USER_TO_2D)) {
            const bool en = fabs(eps - prm.eps_lambda_max) <= prm.near_rel * prm.eps_lambda_max;
            const bool an = fabs(ndw - cth) <= prm.near_rel;
            if ((en && ndw >= cth) || (an && eps < prm.eps_lambda_max) || (en && an)) nr = 1;
          }
        }
      } else if (!in) {
        pre = 1;  // only wall neighbours: h_i >> H_film
      }
    } else if (mi == MAFP_MODEL_2D) {
      H = film_height<T>(i, pos, model, vol, row_ptr, col, (T)prm.alpha_film);
      const T hd = h3d[i];
      if constexpr (sizeof(T) == 4) {
        if (fabsf(H - hd) <= (float)prm.hfilm_band * hd) {
          retake = true;
          const double H64 = film_height<double>(i, pos, model, vol, row_ptr, col, prm.alpha_film);
          pre = (H64 >= (double)hd || (ui & MAFP_USER_TO_3D)) ? 2 : 0;
          if (!(ui & MAFP_USER_TO_3D) && fabs(H64 - (double)hd) <= prm.near_rel * (double)hd) nr = 1;
          H = (T)H64;
        } else {
          pre = (H >= hd || (ui & MAFP_USER_TO_3D)) ? 2 : 0;
        }
      } else {
        pre = (H >= hd || (ui & MAFP_USER_TO_3D)) ? 2 : 0;
        if (!(ui & MAFP_USER_TO_3D) && fabs(H - hd) <= prm.near_rel * hd) nr = 1;
      }
      // tangent frame from the local PCA of the film neighbourhood
      did_pca = true;
      T cov[6];
      int m;
      covariance<T>(i, pos, model, row_ptr, col, cov, &m);
      if constexpr (sizeof(T) == 4) {
        T gap;
        eig3_closed(cov, lam, W, &gap);
      } else {
        double l[3], w[3][3];
        eig3_jacobi(cov, l, w);
        for (int k = 0; k < 3; ++k) {
          lam[k] = l[k];
          for (int r = 0; r < 3; ++r) W[k][r] = w[k][r];
        }
      }
      eps = (lam[0] + lam[1]) > T(0) ? T(2) * lam[2] / (lam[0] + lam[1]) : T(INFINITY);
    }
    if (lane == 0) {
      preflag[i] = pre;
      if (near) near[i] = nr;
      if (nr) inc_ll(&st->n_near);
      if (retake) inc_ll(&st->n_fp64_eigen);
      hfilm[i] = H;
      st4(eig + i, mk4<T>(lam[0], lam[1], lam[2], did_pca ? eps : T(0)));
      st4(frame + 2 * i, did_pca ? mk4<T>(W[0][0], W[0][1], W[0][2], T(0)) : mk4<T>(0, 0, 0, 0));
      st4(frame + 2 * i + 1, did_pca ? mk4<T>(W[2][0], W[2][1], W[2][2], T(0)) : mk4<T>(0, 0, 0, 0));
    }
  }
}

// Sec. 4.3 smoothing, on pre-flags of all particles (order independent).
__global__ void __launch_bounds__(kClsThreads) k_smooth(int64_t n, const uint8_t *model,
                                                        const uint8_t *preflag,
                                                        const uint8_t *last,
                                                        const long long *row_ptr,
                                                        const int32_t *col, uint8_t *flag) {
  const int lane = threadIdx.x & 31;
  const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i = wid; i < n; i += nwarps) {
    uint8_t f = preflag[i];
    if (f != 0 && last[i]) f = 0;
    if (f != 0) {
      const uint8_t target = f == 1 ? MAFP_MODEL_2D : MAFP_MODEL_3D;
      int ok = 0;
      for (long long e = row_ptr[i] + lane; e < row_ptr[i + 1]; e += 32) {
        const int j = col[e];
        if (j != i && (model[j] == target || preflag[j] == f)) ok = 1;
      }
      if (!__any_sync(0xffffffffu, ok)) f = 0;
    }
    if (lane == 0) flag[i] = f;
  }
}

int classify_pca(mafp_ctx *ctx, int64_t n, int32_t dtype, const void *pos_h, const uint8_t *model,
                 const uint8_t *type, const void *normal, const void *vol, const void *h3d,
                 const uint8_t *user, const uint8_t *last, const int64_t *row_ptr,
                 const int32_t *col, uint8_t *flag, uint8_t *preflag, void *eig, void *frame,
                 void *hfilm, uint8_t *near, cudaStream_t s) {
  const int blocks = grid_for(n * 32, kClsThreads, sm_count() * 32);
  const long long *rp = reinterpret_cast<const long long *>(row_ptr);
  if (dtype == MAFP_F64) {
    MAFP_TIMED(ctx, s, "k_classify<double>",
               k_classify<double><<<blocks, kClsThreads, 0, s>>>(
        n, (const double4_16a *)pos_h, model, type, (const double4_16a *)normal, (const double *)vol,
        (const double *)h3d, user, rp, col, preflag, (double4_16a *)eig, (double4_16a *)frame,
        (double *)hfilm, near, ctx->prm, ctx->d_status));
  } else {
    MAFP_TIMED(ctx, s, "k_classify<float>",
               k_classify<float><<<blocks, kClsThreads, 0, s>>>(
        n, (const float4 *)pos_h, model, type, (const float4 *)normal, (const float *)vol,
        (const float *)h3d, user, rp, col, preflag, (float4 *)eig, (float4 *)frame,
        (float *)hfilm, near, ctx->prm, ctx->d_status));
  }
  MAFP_TIMED(ctx, s, "k_smooth",
             k_smooth<<<blocks, kClsThreads, 0, s>>>(n, model, preflag, last, rp, col, flag));
  MAFP_LAUNCH_CHECK(ctx);
  return MAFP_OK;
}

}  // namespace mafp
