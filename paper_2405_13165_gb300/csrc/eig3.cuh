// eig3.cuh -- symmetric 3x3 eigen-decompositions used by the local PCA of
// Sec. 4.1.2: cyclic Jacobi in FP64 and a closed-form FP32 solver.
#pragma once
#include "internal.cuh"

namespace mafp {

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


}  // namespace mafp
