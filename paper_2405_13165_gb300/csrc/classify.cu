// classify.cu -- model-transition detection of Sec. 4 (Alg. 2, Eq. Height,
// Eq. 2Dto3Dcond) and the smoothing of Sec. 4.3.  A group of G lanes per
// particle; lanes stride over the neighbour row and reduce with shuffles.
// The FP32 path takes every decision that lies within a band of its
// threshold again in FP64.
#include <climits>

#include "eig3.cuh"
#include "internal.cuh"

namespace mafp {

constexpr int kClsThreads = 128;

// Thresholds prepared on the host so the FP32 path compares in FP32 only.
struct ClsConst {
  double cth;  // cos(theta*)
  float cth_f, eps_max_f, eps_band_f, angle_band_f, hfilm_band_f;
};

// One pass over the row of particle i: number of same-model neighbours and
// the sum of their coordinates q = (x_j - x_i)/h_i (for the centroid of
// Sec. 4.1.2); for a 2D particle also Eq. Height over its 2D neighbours
// (the same set); for a 3D particle the free-surface / interior neighbour
// flags of the resolution criterion (Sec. 4.1.1, j != i).
template <int G, typename C, typename V, typename TV>
__device__ void row_pass1(int64_t i, const V *pos, const uint8_t *model, const uint8_t *type,
                          const TV *vol, const long long *row_ptr, const int32_t *col, C alpha,
                          int *m_out, C qs[3], C *H_out, int *fs_out, int *in_out) {
  const int lane = threadIdx.x & (G - 1);
  const V xi = ld4(pos + i);
  const uint8_t mi = model[i];
  const C hinv = C(1) / C(xi.w);
  const C api = alpha / C(3.141592653589793);
  C sx = 0, sy = 0, sz = 0, H = 0;
  int m = 0, fs = 0, in = 0;
  for (long long e = row_ptr[i] + lane; e < row_ptr[i + 1]; e += G) {
    const int j = col[e];
    if (model[j] != mi) continue;
    const V xj = ld4(pos + j);
    const C dx = C(xj.x) - C(xi.x), dy = C(xj.y) - C(xi.y), dz = C(xj.z) - C(xi.z);
    sx += dx * hinv;
    sy += dy * hinv;
    sz += dz * hinv;
    ++m;
    if (mi == MAFP_MODEL_2D) {
      if (vol) {
        const C d2 = (dx * dx + dy * dy) + dz * dz;
        const C hj = C(xj.w);
        const C ih2 = C(1) / (hj * hj);
        H += api * ih2 * exp(-alpha * d2 * ih2) * C(vol[j]);
      }
    } else if (j != i) {
      const uint8_t tj = type[j];
      fs |= tj == MAFP_TYPE_FREE_SURFACE;
      in |= tj == MAFP_TYPE_INTERIOR;
    }
  }
  *m_out = group_sum<G>(m);
  qs[0] = group_sum<G>(sx);
  qs[1] = group_sum<G>(sy);
  qs[2] = group_sum<G>(sz);
  *H_out = group_sum<G>(H);
  *fs_out = group_any<G>(fs);
  *in_out = group_any<G>(in);
}

// Scatter matrix sum_j (q_j - q_c)(q_j - q_c)^T over the same-model row (Sec. 4.1.2).
template <int G, typename C, typename V>
__device__ void row_scatter(int64_t i, const V *pos, const uint8_t *model,
                            const long long *row_ptr, const int32_t *col, const C qc[3],
                            C cov[6]) {
  const int lane = threadIdx.x & (G - 1);
  const V xi = ld4(pos + i);
  const uint8_t mi = model[i];
  const C hinv = C(1) / C(xi.w);
  C a[6] = {0, 0, 0, 0, 0, 0};
  for (long long e = row_ptr[i] + lane; e < row_ptr[i + 1]; e += G) {
    const int j = col[e];
    if (model[j] != mi) continue;
    const V xj = ld4(pos + j);
    const C dx = (C(xj.x) - C(xi.x)) * hinv - qc[0];
    const C dy = (C(xj.y) - C(xi.y)) * hinv - qc[1];
    const C dz = (C(xj.z) - C(xi.z)) * hinv - qc[2];
    a[0] += dx * dx; a[1] += dy * dy; a[2] += dz * dz;
    a[3] += dx * dy; a[4] += dx * dz; a[5] += dy * dz;
  }
#pragma unroll
  for (int k = 0; k < 6; ++k) cov[k] = group_sum<G>(a[k]);
}

// FP32 path: the same row in one pass -- the counts, neighbour flags and
// Eq. Height of row_pass1 together with the raw second moments sum_j q_j q_j^T,
// two neighbours gathered ahead per lane; the scatter matrix is formed from
// the moments as sum_j q_j q_j^T - m q_c q_c^T.  (Coordinates are O(1) after
// the scaling by h and the particle sits inside its neighbourhood, so the
// difference loses little; decisions near a threshold are retaken in FP64
// with the two-pass form.)
template <int G, typename V, typename TV>
__device__ void row_one_pass(int64_t i, const V *pos, const uint8_t *model, const uint8_t *type,
                             const TV *vol, const long long *row_ptr, const int32_t *col,
                             float alpha, int *m_out, float cov[6], float qc[3], float *H_out,
                             int *fs_out, int *in_out) {
  constexpr int U = 2;
  const int lane = threadIdx.x & (G - 1);
  const V xi = ld4(pos + i);
  const uint8_t mi = model[i];
  const float hinv = 1.0f / xi.w;
  const float api = alpha / 3.141592653589793f;
  float s[3] = {0, 0, 0}, a[6] = {0, 0, 0, 0, 0, 0}, H = 0;
  int m = 0, fs = 0, in = 0;
  const long long e1 = row_ptr[i + 1];
  for (long long e0 = row_ptr[i] + lane; e0 < e1; e0 += U * G) {
    int js[U];
    V xs[U];
    uint8_t ms[U], ts[U];
#pragma unroll
    for (int u = 0; u < U; ++u) js[u] = e0 + u * G < e1 ? col[e0 + u * G] : -1;
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int j = js[u] >= 0 ? js[u] : (int)i;
      xs[u] = ld4(pos + j);
      ms[u] = model[j];
      ts[u] = type[j];
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int j = js[u];
      if (j < 0 || ms[u] != mi) continue;
      const float dx = xs[u].x - xi.x, dy = xs[u].y - xi.y, dz = xs[u].z - xi.z;
      const float qx = dx * hinv, qy = dy * hinv, qz = dz * hinv;
      s[0] += qx; s[1] += qy; s[2] += qz;
      a[0] += qx * qx; a[1] += qy * qy; a[2] += qz * qz;
      a[3] += qx * qy; a[4] += qx * qz; a[5] += qy * qz;
      ++m;
      if (mi == MAFP_MODEL_2D) {
        if (vol) {
          const float d2 = (dx * dx + dy * dy) + dz * dz;
          const float hj = xs[u].w;
          const float ih2 = 1.0f / (hj * hj);
          H += api * ih2 * expf(-alpha * d2 * ih2) * float(vol[j]);
        }
      } else if (j != i) {
        fs |= ts[u] == MAFP_TYPE_FREE_SURFACE;
        in |= ts[u] == MAFP_TYPE_INTERIOR;
      }
    }
  }
  m = group_sum<G>(m);
#pragma unroll
  for (int k = 0; k < 3; ++k) s[k] = group_sum<G>(s[k]);
#pragma unroll
  for (int k = 0; k < 6; ++k) a[k] = group_sum<G>(a[k]);
  *H_out = group_sum<G>(H);
  *fs_out = group_any<G>(fs);
  *in_out = group_any<G>(in);
  *m_out = m;
  const float im = m > 0 ? 1.0f / (float)m : 0.0f;
  qc[0] = s[0] * im; qc[1] = s[1] * im; qc[2] = s[2] * im;
  cov[0] = a[0] - s[0] * qc[0];
  cov[1] = a[1] - s[1] * qc[1];
  cov[2] = a[2] - s[2] * qc[2];
  cov[3] = a[3] - s[0] * qc[1];
  cov[4] = a[4] - s[0] * qc[2];
  cov[5] = a[5] - s[1] * qc[2];
}

// FP64 PCA of particle i (the retake path): centroid, scatter, Jacobi.
template <int G, typename V>
__device__ void pca64(int64_t i, const V *pos, const uint8_t *model, const uint8_t *type,
                      const long long *row_ptr, const int32_t *col, double lam[3],
                      double W[3][3]) {
  int m, fs, in;
  double qs[3], H;
  row_pass1<G, double>(i, pos, model, type, (const double *)nullptr, row_ptr, col, 0.0, &m, qs,
                       &H, &fs, &in);
  const double im = m > 0 ? 1.0 / m : 0.0;
  const double qc[3] = {qs[0] * im, qs[1] * im, qs[2] * im};
  double cov[6];
  row_scatter<G, double>(i, pos, model, row_ptr, col, qc, cov);
  eig3_jacobi(cov, lam, W);
}

// FP64 film height of particle i (the retake path).
template <int G, typename V, typename TV>
__device__ double hfilm64(int64_t i, const V *pos, const uint8_t *model, const uint8_t *type,
                          const TV *vol, const long long *row_ptr, const int32_t *col,
                          double alpha) {
  int m, fs, in;
  double qs[3], H;
  row_pass1<G, double>(i, pos, model, type, vol, row_ptr, col, alpha, &m, qs, &H, &fs, &in);
  return H;
}

template <typename T, int G>
__global__ void __launch_bounds__(kClsThreads, sizeof(T) == 4 ? 8 : 1) k_classify(
    int64_t n, const vec4_t<T> *pos, const uint8_t *model, const uint8_t *type,
    const vec4_t<T> *normal, const T *vol, const T *h3d, const uint8_t *user,
    const long long *row_ptr, const int32_t *col, uint8_t *preflag, vec4_t<T> *eig,
    vec4_t<T> *frame, T *hfilm, uint8_t *near, mafp_params prm, ClsConst kc, DevStatus *st) {
  using V = vec4_t<T>;
  const int lane = threadIdx.x & (G - 1);
  const int64_t gid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / G;
  const int64_t ngroups = ((int64_t)gridDim.x * blockDim.x) / G;
  const double cth = kc.cth;
  for (int64_t i = gid; i < n; i += ngroups) {
    const uint8_t mi = model[i], ti = type[i], ui = user[i];
    uint8_t pre = 0, nr = 0;
    T lam[3] = {0, 0, 0}, W[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}}, H = 0, eps = 0;
    bool did_pca = false, retake = false;
    if (mi == MAFP_MODEL_2D || ti == MAFP_TYPE_WALL) {
      did_pca = true;
      int m, fs, in;
      T cov[6];
      if constexpr (sizeof(T) == 4) {
        float qc[3];
        row_one_pass<G>(i, pos, model, type, vol, row_ptr, col, (float)prm.alpha_film, &m, cov,
                        qc, &H, &fs, &in);
      } else {
        T qs[3];
        row_pass1<G, T>(i, pos, model, type, vol, row_ptr, col, (T)prm.alpha_film, &m, qs, &H,
                        &fs, &in);
        const T im = m > 0 ? T(1) / T(m) : T(0);
        const T qc[3] = {qs[0] * im, qs[1] * im, qs[2] * im};
        row_scatter<G, T>(i, pos, model, row_ptr, col, qc, cov);
      }
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
      if (mi == MAFP_MODEL_3D) {
        // Alg. 2: resolution criterion, then the PCA criteria or a user request
        if (fs) {
          const V nv = ld4(normal + i);
          const T ndw = fabs(nv.x * W[2][0] + nv.y * W[2][1] + nv.z * W[2][2]);
          bool certain = true;
          if constexpr (sizeof(T) == 4) {
            const bool eps_unsure = fabsf(eps - kc.eps_max_f) <= kc.eps_band_f;
            const bool eps_pass = eps < kc.eps_max_f;
            const bool ang_unsure = fabsf(ndw - kc.cth_f) <= kc.angle_band_f || gap < 1e-2f;
            certain = !(eps_unsure || (eps_pass && ang_unsure));
            if (certain) {
              // FP32 decision away from both thresholds
              pre = ((eps_pass && ndw >= kc.cth_f) || (ui & MAFP_USER_TO_2D)) ? 1 : 0;
            }
          }
          double e64 = eps, d64 = ndw;
          if (!certain) {
            retake = true;
            double l64[3], w64[3][3];
            pca64<G>(i, pos, model, type, row_ptr, col, l64, w64);
            e64 = (l64[0] + l64[1]) > 0.0 ? 2.0 * l64[2] / (l64[0] + l64[1]) : INFINITY;
            d64 = fabs((double)nv.x * w64[2][0] + (double)nv.y * w64[2][1] +
                       (double)nv.z * w64[2][2]);
            for (int k = 0; k < 3; ++k) {
              lam[k] = (T)l64[k];
              for (int r = 0; r < 3; ++r) W[k][r] = (T)w64[k][r];
            }
            eps = (T)e64;
          }
          if (sizeof(T) == 8 || !certain) {
            const bool pass = (e64 < prm.eps_lambda_max) && (d64 >= cth);
            pre = (pass || (ui & MAFP_USER_TO_2D)) ? 1 : 0;
          }
          if ((sizeof(T) == 8 || retake) && !(ui & MAFP_USER_TO_2D)) {
            const bool en = fabs(e64 - prm.eps_lambda_max) <= prm.near_rel * prm.eps_lambda_max;
            const bool an = fabs(d64 - cth) <= prm.near_rel;
            // l2 = l3: w3 is not unique, the eigenvector test has no single answer
            const bool degenerate = ((double)lam[1] - (double)lam[2]) <= 1e-9 * (double)lam[0];
            if ((en && d64 >= cth) || (an && e64 < prm.eps_lambda_max) || (en && an) ||
                (degenerate && e64 < prm.eps_lambda_max))
              nr = 1;
          }
        } else if (!in) {
          pre = 1;  // only wall neighbours: h_i >> H_film
        }
        H = 0;
      } else {
        // Eq. 2Dto3Dcond
        const T hd = h3d[i];
        bool certain = true;
        if constexpr (sizeof(T) == 4) {
          certain = fabsf(H - hd) > kc.hfilm_band_f * hd;
          if (certain) pre = (H >= hd || (ui & MAFP_USER_TO_3D)) ? 2 : 0;
        }
        if (sizeof(T) == 8 || !certain) {
          double H64 = H;
          if (!certain) {
            retake = true;
            H64 = hfilm64<G>(i, pos, model, type, vol, row_ptr, col, prm.alpha_film);
            H = (T)H64;
          }
          pre = (H64 >= (double)hd || (ui & MAFP_USER_TO_3D)) ? 2 : 0;
          if (!(ui & MAFP_USER_TO_3D) && fabs(H64 - (double)hd) <= prm.near_rel * (double)hd)
            nr = 1;
        }
      }
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
template <int G>
__global__ void __launch_bounds__(kClsThreads) k_smooth(int64_t n, const uint8_t *model,
                                                        const uint8_t *preflag,
                                                        const uint8_t *last,
                                                        const long long *row_ptr,
                                                        const int32_t *col, uint8_t *flag) {
  const int lane = threadIdx.x & (G - 1);
  const int64_t gid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / G;
  const int64_t ngroups = ((int64_t)gridDim.x * blockDim.x) / G;
  for (int64_t i = gid; i < n; i += ngroups) {
    uint8_t f = preflag[i];
    if (f != 0 && last[i]) f = 0;
    if (f != 0) {
      const uint8_t target = f == 1 ? MAFP_MODEL_2D : MAFP_MODEL_3D;
      int ok = 0;
      for (long long e = row_ptr[i] + lane; e < row_ptr[i + 1]; e += G) {
        const int j = col[e];
        if (j != i && (model[j] == target || preflag[j] == f)) ok = 1;
      }
      if (!group_any<G>(ok)) f = 0;
    }
    if (lane == 0) flag[i] = f;
  }
}

template <int G>
static int classify_pca_g(mafp_ctx *ctx, int64_t n, int32_t dtype, const void *pos_h,
                          const uint8_t *model, const uint8_t *type, const void *normal,
                          const void *vol, const void *h3d, const uint8_t *user,
                          const uint8_t *last, const int64_t *row_ptr, const int32_t *col,
                          uint8_t *flag, uint8_t *preflag, void *eig, void *frame, void *hfilm,
                          uint8_t *near, cudaStream_t s) {
  static const KernelName n64("k_classify<double,G=%d>", G), n32("k_classify<float,G=%d>", G),
      nsm("k_smooth<G=%d>", G);
  const int blocks = grid_for(n * G, kClsThreads, sm_count() * 32);
  ClsConst kc;
  kc.cth = cos(ctx->prm.theta_star);
  kc.cth_f = (float)kc.cth;
  kc.eps_max_f = (float)ctx->prm.eps_lambda_max;
  kc.eps_band_f = (float)ctx->prm.eps_band;
  kc.angle_band_f = (float)ctx->prm.angle_band;
  kc.hfilm_band_f = (float)ctx->prm.hfilm_band;
  const long long *rp = reinterpret_cast<const long long *>(row_ptr);
  if (dtype == MAFP_F64) {
    MAFP_TIMED(ctx, s, n64.s,
               k_classify<double, G><<<blocks, kClsThreads, 0, s>>>(
                   n, (const double4_16a *)pos_h, model, type, (const double4_16a *)normal,
                   (const double *)vol, (const double *)h3d, user, rp, col, preflag,
                   (double4_16a *)eig, (double4_16a *)frame, (double *)hfilm, near, ctx->prm,
                   kc, ctx->d_status));
  } else {
    MAFP_TIMED(ctx, s, n32.s,
               k_classify<float, G><<<blocks, kClsThreads, 0, s>>>(
                   n, (const float4 *)pos_h, model, type, (const float4 *)normal,
                   (const float *)vol, (const float *)h3d, user, rp, col, preflag, (float4 *)eig,
                   (float4 *)frame, (float *)hfilm, near, ctx->prm, kc, ctx->d_status));
  }
  MAFP_TIMED(ctx, s, nsm.s,
             k_smooth<G><<<blocks, kClsThreads, 0, s>>>(n, model, preflag, last, rp, col, flag));
  MAFP_LAUNCH_CHECK(ctx);
  return MAFP_OK;
}

// Lanes per particle: the context's classify_group (the FP32 sums are reduced
// over the group, so the eigenvalues differ only by rounding; every decision
// near a threshold is retaken in FP64 whatever the group).
int classify_pca(mafp_ctx *ctx, int64_t n, int32_t dtype, const void *pos_h, const uint8_t *model,
                 const uint8_t *type, const void *normal, const void *vol, const void *h3d,
                 const uint8_t *user, const uint8_t *last, const int64_t *row_ptr,
                 const int32_t *col, uint8_t *flag, uint8_t *preflag, void *eig, void *frame,
                 void *hfilm, uint8_t *near, cudaStream_t s) {
  switch (ctx->tune.classify_group) {
    case 1:
      return classify_pca_g<1>(ctx, n, dtype, pos_h, model, type, normal, vol, h3d, user, last,
                               row_ptr, col, flag, preflag, eig, frame, hfilm, near, s);
    case 2:
      return classify_pca_g<2>(ctx, n, dtype, pos_h, model, type, normal, vol, h3d, user, last,
                               row_ptr, col, flag, preflag, eig, frame, hfilm, near, s);
    case 4:
      return classify_pca_g<4>(ctx, n, dtype, pos_h, model, type, normal, vol, h3d, user, last,
                               row_ptr, col, flag, preflag, eig, frame, hfilm, near, s);
    case 16:
      return classify_pca_g<16>(ctx, n, dtype, pos_h, model, type, normal, vol, h3d, user, last,
                                row_ptr, col, flag, preflag, eig, frame, hfilm, near, s);
    default:
      return classify_pca_g<8>(ctx, n, dtype, pos_h, model, type, normal, vol, h3d, user, last,
                               row_ptr, col, flag, preflag, eig, frame, hfilm, near, s);
  }
}

}  // namespace mafp
