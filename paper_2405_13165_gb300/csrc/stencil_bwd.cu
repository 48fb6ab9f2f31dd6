// stencil_bwd.cu -- adjoint of (build_stencils, apply_ops) with respect to the
// particle positions, recomputing the moment matrix and its Cholesky factor
// per particle (no stored factors).
//
// For one row i with c_jk = w_j p_j . lambda_k, (sum_j w_j p_j p_j^T) lambda_k = b_k
// and gbar_jk = dL/dc_jk = sum_f gout[i][f][k] (u_j - u_i):
//   lbar_k = sum_j gbar_jk w_j p_j,  mu_k = A^-1 lbar_k,
//   s_jk = p_j . lambda_k,  t_jk = p_j . mu_k,
//   wbar_j = sum_k (gbar_jk - t_jk) s_jk,
//   pbar_j = w_j sum_k (gbar_jk lambda_k - s_jk mu_k - t_jk lambda_k),
// then through p(q) and W(|q|) to q_j = (x_j - x_i)/h_i, scattered to x_j and
// x_i (atomic adds).  The unscaled right-hand sides of the forward kernel are
// used; the 1/h and 1/h^2 output factors are folded into gbar.
//
// Film rows: the tangent frame (t1, t2, n = w3) is the local PCA of Sec. 4.1.2
// over the same-model part of S_i, so it moves with the positions too.  The
// outputs do not change when (t1, t2) turn inside the plane; only n matters.
// With tbar_k = dL/dt_k at fixed n (through xi = d.t1/h, eta = d.t2/h and the
// world-coordinate gradient c^xi t1 + c^eta t2), turning the frame with n and
// the first-order perturbation of the eigenvector w3 of the scatter matrix
// Ps = sum_j z_j z_j^T (z_j = y_j - y_c, y_j = (x_j - x_i)/h) give
//   dL/dy_j = sum_k beta_k (t_k (n.z_j) + n (t_k.z_j)),  beta_k = (tbar_k.n)/(l_k - l3),
// with l_k = t_k^T Ps t_k (Rayleigh quotients in the given frame).  The gradient
// pass also sums n.tbar_k and the neighbours' frame coordinates and their
// squares; a third pass over the row scatters the term.
#include "internal.cuh"
#include "stencil_common.cuh"

namespace mafp {

// dL/dx of one particle into its 4-wide gpos record: one vector atomic for
// FP32 (16-byte aligned records), three scalar ones for FP64.
template <typename T>
__device__ __forceinline__ void add_xyz(T *p, T x, T y, T z);
template <>
__device__ __forceinline__ void add_xyz<float>(float *p, float x, float y, float z) {
  atomicAdd(reinterpret_cast<float4 *>(p), make_float4(x, y, z, 0.0f));
}
template <>
__device__ __forceinline__ void add_xyz<double>(double *p, double x, double y, double z) {
  atomicAdd(p, x);
  atomicAdd(p + 1, y);
  atomicAdd(p + 2, z);
}

// neighbours a lane gathers ahead of use in the moment / lbar pass and the gradient pass
constexpr int kGradGatherA = 2, kGradGatherC = 2;
// ring depth of the streamed passes (entries in flight per lane)
constexpr int kGradRing = 2;

// Returns 0 done, 1 no gradient (deficient), 2 queued for the FP64 redo.
// RING (FP32 storage and arithmetic): the passes over the row stream the
// neighbour records through the block's shared-memory ring (stream_row)
// instead of gathering a few entries at a time into registers.
template <typename TS, typename C, int M, int G, bool QUEUE, bool RING = false>
__device__ int grad_particle(int64_t i, const vec4_t<TS> *pos, const uint8_t *model,
                             const vec4_t<TS> *frame, const long long *row_ptr,
                             const int32_t *col, const vec4_t<TS> *fields,
                             const vec4_t<TS> *gout, TS *gpos, const StParams<C> &sp, C *sm,
                             float4 *ring = nullptr) {
  constexpr int NA = Basis<M>::NA, NR = Basis<M>::NR;
  constexpr int VA = pad_to(NA, G), VR = pad_to(NR * M, G);
  using V = vec4_t<TS>;
  const int lane = threadIdx.x & (G - 1);
  const unsigned gm = group_mask<G>();
  const V xi = ld4(pos + i);
  const uint8_t mi = model[i];
  const C hinv = C(1) / C(xi.w);
  C t1[3] = {0, 0, 0}, t2[3] = {0, 0, 0}, nv[3] = {0, 0, 0};
  if constexpr (M == 6) {
    const V f1 = ld4(frame + 2 * i), f3 = ld4(frame + 2 * i + 1);
    t1[0] = C(f1.x); t1[1] = C(f1.y); t1[2] = C(f1.z);
    nv[0] = C(f3.x); nv[1] = C(f3.y); nv[2] = C(f3.z);
    t2[0] = nv[1] * t1[2] - nv[2] * t1[1];
    t2[1] = nv[2] * t1[0] - nv[0] * t1[2];
    t2[2] = nv[0] * t1[1] - nv[1] * t1[0];
  }
  const long long b = row_ptr[i], e1 = row_ptr[i + 1];
  // per-operator output scale of the forward kernel: gradient 1/h, Laplacian 1/h^2
  const C h2inv = hinv * hinv;
  const V fi = ld4(fields + i);
  // gout of row i; 3D rows fold the output scale into it (gs = gout * (1/h, 1/h,
  // 1/h, 1/h^2) per field), film rows keep it unscaled for the frame terms
  C gs[4][4];
#pragma unroll
  for (int f = 0; f < 4; ++f) {
    const V g = ld4(gout + 4 * i + f);
    const C sg = M == 10 ? hinv : C(1), sl = M == 10 ? h2inv : C(1);
    gs[f][0] = C(g.x) * sg; gs[f][1] = C(g.y) * sg; gs[f][2] = C(g.z) * sg; gs[f][3] = C(g.w) * sl;
  }
  // gbar (scaled) of one neighbour, in the basis' operator order; g4 = the
  // unscaled sum_f gout[i][f][.] du_f of film rows
  auto gbar = [&](const V &fj, C (&gb)[NR], C (&g4)[4]) {
    const C du[4] = {C(fj.x) - C(fi.x), C(fj.y) - C(fi.y), C(fj.z) - C(fi.z), C(fj.w) - C(fi.w)};
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      C v = gs[0][c] * du[0];
#pragma unroll
      for (int f = 1; f < 4; ++f) v = fma(gs[f][c], du[f], v);
      g4[c] = v;
    }
    if constexpr (M == 10) {
      gb[0] = g4[0]; gb[1] = g4[1]; gb[2] = g4[2]; gb[3] = g4[3];
    } else {
      gb[0] = (g4[0] * t1[0] + g4[1] * t1[1] + g4[2] * t1[2]) * hinv;
      gb[1] = (g4[0] * t2[0] + g4[1] * t2[1] + g4[2] * t2[2]) * hinv;
      gb[2] = g4[3] * h2inv;
    }
  };
  // ---- one pass: moments A = sum_j w_j p_j p_j^T and lbar_k = sum_j gbar_jk w_j p_j
  // (gbar depends on the fields only, so it needs no solution yet)
  constexpr int VM = pad_to(Moments<M>::N, G);
  C A[VM];   // the distinct moments
#pragma unroll
  for (int k = 0; k < VM; ++k) A[k] = C(0);
  C R[VR];
#pragma unroll
  for (int k = 0; k < VR; ++k) R[k] = C(0);
  // lbar is linear in the field differences: the pass sums B_f = sum_j w_j
  // du_jf p_j and lbar_k = sum_f gout[i][f][k] B_f (scaled as gbar) follows
  C Bf[4 * M];
#pragma unroll
  for (int k = 0; k < 4 * M; ++k) Bf[k] = C(0);
  int cnt = 0;
  auto pass1 = [&](const V &xj, const V &fj, int, bool ok) {
    C p[M];
    C w = basis_at<M, C>(xi, ok ? xj : xi, hinv, t1, t2, sp, p);
    w = ok ? w : C(0);   // other model / past the row end: contributes exact zeros
    cnt += ok ? 1 : 0;
    add_moments<M, C, VM>(A, w, p);
    const V fv = ok ? fj : fi;
    const C wdu[4] = {w * (C(fv.x) - C(fi.x)), w * (C(fv.y) - C(fi.y)),
                      w * (C(fv.z) - C(fi.z)), w * (C(fv.w) - C(fi.w))};
#pragma unroll
    for (int f = 0; f < 4; ++f)
#pragma unroll
      for (int r = 0; r < M; ++r) Bf[f * M + r] += wdu[f] * p[r];
  };
  if constexpr (RING) {
    stream_row<kGradRing, G, true>(b, e1, mi, col, pos, model, fields, ring, pass1);
  } else {
    for (long long e0 = b + lane; e0 < e1; e0 += kGradGatherA * G) {
      V xs[kGradGatherA], fs[kGradGatherA];
      int js[kGradGatherA];
      bool oks[kGradGatherA];
      gather_row_f<kGradGatherA, G>(e0, e1, i, mi, col, pos, model, fields, xs, fs, js, oks);
#pragma unroll
      for (int u = 0; u < kGradGatherA; ++u) pass1(xs[u], fs[u], js[u], oks[u]);
    }
  }
#pragma unroll
  for (int r = 0; r < M; ++r) {
    C g4[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      C v = gs[0][c] * Bf[r];
#pragma unroll
      for (int f = 1; f < 4; ++f) v = fma(gs[f][c], Bf[f * M + r], v);
      g4[c] = v;
    }
    if constexpr (M == 10) {
#pragma unroll
      for (int c = 0; c < 4; ++c) R[c * M + r] = g4[c];
    } else {
      R[0 * M + r] = (g4[0] * t1[0] + g4[1] * t1[1] + g4[2] * t1[2]) * hinv;
      R[1 * M + r] = (g4[0] * t2[0] + g4[1] * t2[1] + g4[2] * t2[2]) * hinv;
      R[2 * M + r] = g4[3] * h2inv;
    }
  }
  cnt = group_sum<G>(cnt);
  reduce_scatter<G, VM>(A);
  reduce_scatter<G, VR>(R);
  __syncwarp(gm);
#pragma unroll
  for (int k = 0; k < VM / G; ++k) sm[lane * (VM / G) + k] = A[k];
  __syncwarp(gm);
  C L[NA];
  constexpr MomentTable<M> MT = Moments<M>::T;
#pragma unroll
  for (int k = 0; k < NA; ++k) L[k] = sm[MT.idx[k]];
  __syncwarp(gm);
#pragma unroll
  for (int k = 0; k < VR / G; ++k) sm[lane * (VR / G) + k] = R[k];
  __syncwarp(gm);
  C tr = 0;
#pragma unroll
  for (int r = 0; r < M; ++r) tr += L[pk(r, r)];
  C invd[M], pmin, pmax;
  const bool ok = (cnt >= M) && cholesky<M, C>(L, invd, sp.piv_tol_rel * tr, pmin, pmax);
  const C cond = (pmax / pmin) * (pmax / pmin);
  if (!ok || (QUEUE && !(cond <= sp.cond_max))) return (QUEUE && cnt >= M) ? 2 : 1;
  C *Ls = sm + StSmem<M, G>::SCR;
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < NA; ++k) Ls[k] = L[k];
  }
  __syncwarp(gm);
  C lam[NR][M];
#pragma unroll
  for (int k = 0; k < NR; ++k) {
    C bb[M];
#pragma unroll
    for (int r = 0; r < M; ++r) bb[r] = rhs<M, C>(k, r);
    chol_solve_s<M, C>(Ls, invd, bb, lam[k]);
  }
  // ---- mu_k = A^-1 lbar_k
  C mu[NR][M];
#pragma unroll
  for (int k = 0; k < NR; ++k) {
    C lb[M];
#pragma unroll
    for (int r = 0; r < M; ++r) lb[r] = sm[k * M + r];
    chol_solve_s<M, C>(Ls, invd, lb, mu[k]);
  }
  __syncwarp(gm);
  // ---- pass 2: wbar, pbar -> dL/dx_j (scattered) and -sum for x_i
  const C a2 = C(-2) * sp.alpha * sp.inv_den;  // W'(s)/s = a2 exp(-alpha s^2)
  C acc_i[3] = {0, 0, 0};
  C tn1 = 0, tn2 = 0;   // film rows: n . dL/dt1 and n . dL/dt2 at fixed n
  // film rows: sums of the frame coordinates (xi, eta, zeta) = y.(t1, t2, n) of
  // the neighbours and of their squares (the PCA's Rayleigh quotients)
  C sc[3] = {0, 0, 0}, sq[3] = {0, 0, 0};
  auto pass2 = [&](const V &xj, const V &fj, int j, bool ok) {
    if (!ok || j == i) return;
    C p[M], gb[NR], g4[4];
    const C dx = C(xj.x) - C(xi.x), dy = C(xj.y) - C(xi.y), dz = C(xj.z) - C(xi.z);
    // one exponential serves W and W' (W'(s)/s = a2 exp(-alpha s^2))
    C ew;
    const C w = basis_at<M, C>(xi, xj, hinv, t1, t2, sp, p, &ew);
    const C s2 = ((dx * dx + dy * dy) + dz * dz) * (hinv * hinv);
    const C dws = s2 <= C(1) ? a2 * ew : C(0);
    gbar(fj, gb, g4);
    // pbar = w sum_k ((gbar_k - t_k) lambda_k - s_k mu_k); pbar_0 is not needed
    // (d p_0 / d q = 0) and the factor w is applied to the gradient below.
    // Every sum is a chain of fused multiply-adds (p_0 = 1 starts the dot products).
    C wbar = 0, pbar[M], s01[2] = {0, 0};
#pragma unroll
    for (int k = 0; k < NR; ++k) {
      C s = lam[k][0], t = mu[k][0];
#pragma unroll
      for (int r = 1; r < M; ++r) {
        s = fma(p[r], lam[k][r], s);
        t = fma(p[r], mu[k][r], t);
      }
      if (k < 2) s01[k] = s;
      const C a = gb[k] - t;
      wbar = fma(a, s, wbar);
#pragma unroll
      for (int r = 1; r < M; ++r) {
        pbar[r] = k == 0 ? a * lam[k][r] : fma(a, lam[k][r], pbar[r]);
        pbar[r] = fma(-s, mu[k][r], pbar[r]);
      }
    }
    const C wq = dws * wbar;
    C d[3];
    if constexpr (M == 10) {
      const C qx = dx * hinv, qy = dy * hinv, qz = dz * hinv;
      const C wh = w * hinv, wqh = wq * hinv;
      const C gx = fma(C(2) * qx, pbar[4], fma(qy, pbar[7], fma(qz, pbar[8], pbar[1])));
      const C gy = fma(C(2) * qy, pbar[5], fma(qx, pbar[7], fma(qz, pbar[9], pbar[2])));
      const C gz = fma(C(2) * qz, pbar[6], fma(qx, pbar[8], fma(qy, pbar[9], pbar[3])));
      d[0] = fma(wqh, qx, wh * gx);
      d[1] = fma(wqh, qy, wh * gy);
      d[2] = fma(wqh, qz, wh * gz);
    } else {
      const C xi_ = p[1], et_ = p[2];
      // xbh, ebh = dL/dxi, dL/deta (with w) over h
      const C wh = w * hinv, wqh2 = wq * h2inv;
      const C xbh = wh * fma(C(2) * xi_, pbar[3], fma(et_, pbar[4], pbar[1]));
      const C ebh = wh * fma(xi_, pbar[4], fma(C(2) * et_, pbar[5], pbar[2]));
      d[0] = fma(xbh, t1[0], fma(ebh, t2[0], wqh2 * dx));
      d[1] = fma(xbh, t1[1], fma(ebh, t2[1], wqh2 * dy));
      d[2] = fma(xbh, t1[2], fma(ebh, t2[2], wqh2 * dz));
      // the frame through xi, eta and through c^xi t1 + c^eta t2 (c^xi = w s_0 / h);
      // only the normal components of dL/dt_k are needed
      const C dn = dx * nv[0] + dy * nv[1] + dz * nv[2];
      const C gn = g4[0] * nv[0] + g4[1] * nv[1] + g4[2] * nv[2];
      tn1 = fma(xbh, dn, fma(wh * s01[0], gn, tn1));
      tn2 = fma(ebh, dn, fma(wh * s01[1], gn, tn2));
      const C ze = dn * hinv;
      sc[0] += xi_; sc[1] += et_; sc[2] += ze;
      sq[0] += xi_ * xi_; sq[1] += et_ * et_; sq[2] += ze * ze;
    }
    add_xyz<TS>(gpos + 4 * (int64_t)j, TS(d[0]), TS(d[1]), TS(d[2]));
#pragma unroll
    for (int a = 0; a < 3; ++a) acc_i[a] -= d[a];
  };
  if constexpr (RING) {
    stream_row<kGradRing, G, true>(b, e1, mi, col, pos, model, fields, ring, pass2);
  } else {
    for (long long e0 = b + lane; e0 < e1; e0 += kGradGatherC * G) {
      V xs[kGradGatherC], fs[kGradGatherC];
      int js[kGradGatherC];
      bool oks[kGradGatherC];
      gather_row_f<kGradGatherC, G>(e0, e1, i, mi, col, pos, model, fields, xs, fs, js, oks);
#pragma unroll
      for (int u = 0; u < kGradGatherC; ++u) pass2(xs[u], fs[u], js[u], oks[u]);
    }
  }
  if constexpr (M == 6) {
    // ---- pass 3 (film rows): the PCA frame's dependence on the positions.
    // With the frame coordinates' sums from pass 2, the centroid is
    // y_c = xc t1 + ec t2 + zc n and l_k - l3 follow from the Rayleigh
    // quotients; one more pass over the row scatters the term.
    tn1 = group_sum<G>(tn1);
    tn2 = group_sum<G>(tn2);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      sc[a] = group_sum<G>(sc[a]);
      sq[a] = group_sum<G>(sq[a]);
    }
    const C inv_m = C(1) / C(cnt);
    const C xc = sc[0] * inv_m, ec = sc[1] * inv_m, zc = sc[2] * inv_m;
    const C l3 = sq[2] - sc[2] * zc;
    const C g1 = (sq[0] - sc[0] * xc) - l3, g2 = (sq[1] - sc[1] * ec) - l3;
    const C be1 = g1 > C(0) ? tn1 / g1 : C(0);
    const C be2 = g2 > C(0) ? tn2 / g2 : C(0);
    // dL/dx_j = ((be1 t1 + be2 t2) (n.z_j) + n (be1 t1.z_j + be2 t2.z_j)) / h
    C av[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) av[a] = (be1 * t1[a] + be2 * t2[a]) * hinv;
    const C bn1 = be1 * hinv, bn2 = be2 * hinv;
    auto pass3 = [&](const V &xj, const V &, int j, bool ok) {
      if (!ok || j == i) return;
      const C dx = C(xj.x) - C(xi.x), dy = C(xj.y) - C(xi.y), dz = C(xj.z) - C(xi.z);
      const C zn = (dx * nv[0] + dy * nv[1] + dz * nv[2]) * hinv - zc;
      const C z1 = (dx * t1[0] + dy * t1[1] + dz * t1[2]) * hinv - xc;
      const C z2 = (dx * t2[0] + dy * t2[1] + dz * t2[2]) * hinv - ec;
      const C tz = bn1 * z1 + bn2 * z2;
      C d[3];
#pragma unroll
      for (int a = 0; a < 3; ++a) d[a] = av[a] * zn + nv[a] * tz;
      add_xyz<TS>(gpos + 4 * (int64_t)j, TS(d[0]), TS(d[1]), TS(d[2]));
#pragma unroll
      for (int a = 0; a < 3; ++a) acc_i[a] -= d[a];
    };
    if constexpr (RING) {
      stream_row<kGradRing, G, false>(b, e1, mi, col, pos, model, nullptr, ring, pass3);
    } else {
      constexpr int U = 4;
      for (long long e0 = b + lane; e0 < e1; e0 += U * G) {
        V xs[U];
        bool oks[U];
        gather_row<U, G>(e0, e1, i, mi, col, pos, model, xs, oks);
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const long long e = e0 + (long long)u * G;
          pass3(xs[u], xs[u], oks[u] ? col[e] : -1, oks[u]);
        }
      }
    }
  }
#pragma unroll
  for (int a = 0; a < 3; ++a) acc_i[a] = group_sum<G>(acc_i[a]);
  if (lane == 0) add_xyz<TS>(gpos + 4 * i, TS(acc_i[0]), TS(acc_i[1]), TS(acc_i[2]));
  return 0;
}

template <typename TS, typename C, int M, int G, bool QUEUE>
__global__ void __launch_bounds__(kStThreads, sizeof(C) == 4 ? (M == 10 ? 3 : 4) : 1) k_stencil_grad(
    int64_t n, const vec4_t<TS> *pos, const uint8_t *model, const vec4_t<TS> *frame,
    const long long *row_ptr, const int32_t *col, const vec4_t<TS> *fields,
    const vec4_t<TS> *gout, TS *gpos, StParams<C> sp, DevStatus *st, int32_t *queue) {
  constexpr int SMG = StSmem<M, G>::PER_GROUP;
  // 3D rows stream their neighbours through a shared-memory ring (measured on
  // the 1M jet cloud: 1.41 -> 1.34 ms with 2 entries in flight; 1.50 / 1.34 /
  // 1.51 ms with 1 / 3 / 4).  Film rows keep the register gathers: with the
  // ring their instance spills at its 128-register bound (0.55 -> 0.56-0.62 ms).
  constexpr bool RING = sizeof(TS) == 4 && sizeof(C) == 4 && M == 10;
  __shared__ C smem[(kStThreads / G) * SMG];
  // ring of the streamed passes: kGradRing slots x (position, field) per thread
  __shared__ float4 ring[RING ? kGradRing * 2 * kStThreads : 1];
  C *sm = smem + (threadIdx.x / G) * SMG;
  const int lane = threadIdx.x & (G - 1);
  const int64_t gid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / G;
  const int64_t ngroups = ((int64_t)gridDim.x * blockDim.x) / G;
  const uint8_t want = M == 10 ? MAFP_MODEL_3D : MAFP_MODEL_2D;
  for (int64_t i = gid; i < n; i += ngroups) {
    if (model[i] != want) continue;
    const int res = grad_particle<TS, C, M, G, QUEUE, RING>(i, pos, model, frame, row_ptr, col,
                                                           fields, gout, gpos, sp, sm, ring);
    if (res == 2 && lane == 0) queue[atomicAdd(&st->fallback_count, 1)] = (int32_t)i;
  }
}

// FP64 redo of the queued rows of one model (FP32 storage).
template <int M, int G>
__global__ void __launch_bounds__(kStThreads) k_stencil_grad_redo(
    const float4 *pos, const uint8_t *model, const float4 *frame, const long long *row_ptr,
    const int32_t *col, const float4 *fields, const float4 *gout, float *gpos,
    StParams<double> sp, const DevStatus *st, const int32_t *queue) {
  constexpr int SMG = StSmem<M, G>::PER_GROUP;
  __shared__ double smem[(kStThreads / G) * SMG];
  double *sm = smem + (threadIdx.x / G) * SMG;
  const int64_t gid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / G;
  const int64_t ngroups = ((int64_t)gridDim.x * blockDim.x) / G;
  const int nq = st->fallback_count;
  const uint8_t want = M == 10 ? MAFP_MODEL_3D : MAFP_MODEL_2D;
  for (int64_t q = gid; q < nq; q += ngroups) {
    const int64_t i = queue[q];
    if (model[i] != want) continue;
    grad_particle<float, double, M, G, false>(i, pos, model, frame, row_ptr, col, fields, gout,
                                              gpos, sp, sm);
  }
}

__global__ void k_reset_grad_queue(DevStatus *st) { st->fallback_count = 0; }

template <typename TS, typename C, int M, int G, bool QUEUE>
static void launch_grad_g(mafp_ctx *ctx, cudaStream_t s, int64_t n, const void *pos_h,
                          const uint8_t *model, const void *frame, const long long *rp,
                          const int32_t *col, const void *fields, const void *gout, void *gpos,
                          const StParams<C> &sp) {
  using V = vec4_t<TS>;
  static const KernelName name("k_stencil_grad<%s,M=%d,G=%d>", sizeof(TS) == 4 ? "f32" : "f64",
                               M, G);
  MAFP_TIMED(ctx, s, name.s,
             (k_stencil_grad<TS, C, M, G, QUEUE><<<grid_for(n * G, kStThreads, sm_count() * 64),
                                                   kStThreads, 0, s>>>(
                 n, (const V *)pos_h, model, (const V *)frame, rp, col, (const V *)fields,
                 (const V *)gout, (TS *)gpos, sp, ctx->d_status, ctx->fallback)));
}

// Group sizes: grad3d_group for 3D particles (at least 8 in FP64, where the
// 2- and 4-lane instances would spill their registers), grad2d_group for 2D ones.
template <typename TS, typename C, bool QUEUE>
static void launch_grad(mafp_ctx *ctx, cudaStream_t s, int64_t n, const void *pos_h,
                        const uint8_t *model, const void *frame, const long long *rp,
                        const int32_t *col, const void *fields, const void *gout, void *gpos,
                        const StParams<C> &sp) {
  switch (ctx->tune.grad3d_group) {
    case 2:
      if constexpr (sizeof(TS) == 4) {
        launch_grad_g<TS, C, 10, 2, QUEUE>(ctx, s, n, pos_h, model, frame, rp, col, fields, gout, gpos, sp);
        break;
      }
      [[fallthrough]];
    case 4:
      if constexpr (sizeof(TS) == 4) {
        launch_grad_g<TS, C, 10, 4, QUEUE>(ctx, s, n, pos_h, model, frame, rp, col, fields, gout, gpos, sp);
        break;
      }
      [[fallthrough]];
    case 8: launch_grad_g<TS, C, 10, 8, QUEUE>(ctx, s, n, pos_h, model, frame, rp, col, fields, gout, gpos, sp); break;
    case 16: launch_grad_g<TS, C, 10, 16, QUEUE>(ctx, s, n, pos_h, model, frame, rp, col, fields, gout, gpos, sp); break;
    default: launch_grad_g<TS, C, 10, 32, QUEUE>(ctx, s, n, pos_h, model, frame, rp, col, fields, gout, gpos, sp); break;
  }
  switch (ctx->tune.grad2d_group) {
    case 1: launch_grad_g<TS, C, 6, 1, QUEUE>(ctx, s, n, pos_h, model, frame, rp, col, fields, gout, gpos, sp); break;
    case 2: launch_grad_g<TS, C, 6, 2, QUEUE>(ctx, s, n, pos_h, model, frame, rp, col, fields, gout, gpos, sp); break;
    case 4: launch_grad_g<TS, C, 6, 4, QUEUE>(ctx, s, n, pos_h, model, frame, rp, col, fields, gout, gpos, sp); break;
    case 16: launch_grad_g<TS, C, 6, 16, QUEUE>(ctx, s, n, pos_h, model, frame, rp, col, fields, gout, gpos, sp); break;
    default: launch_grad_g<TS, C, 6, 8, QUEUE>(ctx, s, n, pos_h, model, frame, rp, col, fields, gout, gpos, sp); break;
  }
}

int build_stencils_backward(mafp_ctx *ctx, int64_t n, int32_t dtype, const void *pos_h,
                            const uint8_t *model, const void *frame, const int64_t *row_ptr,
                            const int32_t *col, const void *fields, const void *gout, void *gpos,
                            cudaStream_t s) {
  const long long *rp = reinterpret_cast<const long long *>(row_ptr);
  const size_t real = dtype == MAFP_F64 ? sizeof(double) : sizeof(float);
  MAFP_CUDA_TRY(ctx, cudaMemsetAsync(gpos, 0, (size_t)n * 4 * real, s));
  if (dtype == MAFP_F64) {
    launch_grad<double, double, false>(ctx, s, n, pos_h, model, frame, rp, col, fields, gout,
                                       gpos, make_params<double>(ctx->prm, 1e-12));
    MAFP_LAUNCH_CHECK(ctx);
    return MAFP_OK;
  }
  MAFP_TIMED(ctx, s, "k_reset_grad_queue", k_reset_grad_queue<<<1, 1, 0, s>>>(ctx->d_status));
  launch_grad<float, float, true>(ctx, s, n, pos_h, model, frame, rp, col, fields, gout, gpos,
                                  make_params<float>(ctx->prm, 1e-6));
  const StParams<double> sp64 = make_params<double>(ctx->prm, 1e-12);
  const int sms = sm_count();
  MAFP_TIMED(ctx, s, "k_stencil_grad_redo<10>",
             (k_stencil_grad_redo<10, 8><<<sms * 16, kStThreads, 0, s>>>(
                 (const float4 *)pos_h, model, (const float4 *)frame, rp, col,
                 (const float4 *)fields, (const float4 *)gout, (float *)gpos, sp64,
                 ctx->d_status, ctx->fallback)));
  MAFP_TIMED(ctx, s, "k_stencil_grad_redo<6>",
             (k_stencil_grad_redo<6, 8><<<sms * 4, kStThreads, 0, s>>>(
                 (const float4 *)pos_h, model, (const float4 *)frame, rp, col,
                 (const float4 *)fields, (const float4 *)gout, (float *)gpos, sp64,
                 ctx->d_status, ctx->fallback)));
  MAFP_LAUNCH_CHECK(ctx);
  return MAFP_OK;
}

}  // namespace mafp
