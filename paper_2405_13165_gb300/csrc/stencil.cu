// stencil.cu -- GFDM stencils of Eq. GFDM_Definition (Sec. 2.3), order 2.
//
// One group of G lanes per particle (G = 32 for 3D rows of ~180 entries, 8 for
// 2D rows of ~40).  Lanes stride over the row, accumulate the packed moment
// matrix A = sum_j w_j p_j p_j^T, reduce it with a reduce-scatter of shuffles,
// factor it (Cholesky) and solve for the four right-hand sides in every lane.
// FP32 path: one refinement step with the residual b - sum_j c_j p_j of the
// rounded coefficients; particles whose Cholesky pivots are too small or whose
// condition estimate exceeds cond_fp64 are queued and redone in FP64.
#include "internal.cuh"
#include "stencil_common.cuh"

namespace mafp {

__global__ void k_reset_queue(DevStatus *st) { st->fallback_count = 0; }

// Per-lane cache of (q, w) for the refinement and coefficient passes (FP32
// path): 176 entries per 3D row, 48 per film row; entries beyond it are
// gathered and recomputed as in the first pass.
template <typename C, int M, int G>
struct StCache {
  static constexpr int KC = sizeof(C) == 4 ? (M == 10 ? 176 : 48) / G : 0;
  static constexpr int BYTES = (kStThreads / G) * KC * G * (int)sizeof(float4);
  static constexpr int SMEM = BYTES + (kStThreads / G) * StSmem<M, G>::PER_GROUP * (int)sizeof(C);
};

// neighbours a lane gathers ahead of use: 4 for 3D rows (long rows, the loads
// in flight together), 2 for film rows
template <int M> constexpr int kGatherU = M == 10 ? 4 : 2;
constexpr int kGatherR = 2;   // the same in the refinement pass (more live registers)

// Process particle i with a group of G lanes.  Returns (through *result)
//  0 = written, 1 = deficient (zeros written), 2 = queued for FP64.
template <typename TS, typename C, int M, int G, bool REFINE, bool QUEUE, int KC = 0>
__device__ void stencil_particle(int64_t i, const vec4_t<TS> *pos, const uint8_t *model,
                                 const vec4_t<TS> *frame, const long long *row_ptr,
                                 const int32_t *col, vec4_t<TS> *coef, const StParams<C> &sp,
                                 C *sm /* per-group scratch, >= pad_to(NR*M or NA, G) */,
                                 int *result, float *cond_out, float4 *qw = nullptr) {
  constexpr int NA = Basis<M>::NA, NR = Basis<M>::NR;
  constexpr int VA = pad_to(NA, G), VR = pad_to(NR * M, G);
  using V = vec4_t<TS>;
  const int lane = threadIdx.x & (G - 1);
  const unsigned gm = group_mask<G>();
  const V xi = ld4(pos + i);
  const uint8_t mi = model[i];
  const C hinv = C(1) / C(xi.w);
  C t1[3] = {0, 0, 0}, t2[3] = {0, 0, 0};
  if constexpr (M == 6) {
    const V f1 = ld4(frame + 2 * i), f3 = ld4(frame + 2 * i + 1);
    t1[0] = C(f1.x); t1[1] = C(f1.y); t1[2] = C(f1.z);
    const C n0 = C(f3.x), n1 = C(f3.y), n2 = C(f3.z);
    t2[0] = n1 * t1[2] - n2 * t1[1];
    t2[1] = n2 * t1[0] - n0 * t1[2];
    t2[2] = n0 * t1[1] - n1 * t1[0];
  }
  const long long b = row_ptr[i], e1 = row_ptr[i + 1];
  // ---- moments (the distinct ones)
  constexpr int VM = pad_to(Moments<M>::N, G);
  C A[VM];
#pragma unroll
  for (int k = 0; k < VM; ++k) A[k] = C(0);
  int cnt = 0;
  int kk = 0;   // this lane's running entry index: entry b + lane + kk G
  for (long long e0 = b + lane; e0 < e1; e0 += kGatherU<M> * G, kk += kGatherU<M>) {
    V xs[kGatherU<M>];
    bool oks[kGatherU<M>];
    gather_row<kGatherU<M>, G>(e0, e1, i, mi, col, pos, model, xs, oks);
#pragma unroll
    for (int u = 0; u < kGatherU<M>; ++u) {
      C p[M];
      C w = basis_at<M, C>(xi, xs[u], hinv, t1, t2, sp, p);
      w = oks[u] ? w : C(0);   // other model / past the row end: contributes exact zeros
      cnt += oks[u] ? 1 : 0;
      if constexpr (KC > 0) {
        // keep (q, w) for the later passes: they rebuild p without a gather
        if (kk + u < KC) qw[(kk + u) * G + lane] = make_float4(p[1], p[2], M == 10 ? p[3] : 0.f, w);
      }
      add_moments<M, C, VM>(A, w, p);
    }
  }
  cnt = group_sum<G>(cnt);
  reduce_scatter<G, VM>(A);
  __syncwarp(gm);
#pragma unroll
  for (int k = 0; k < VM / G; ++k) sm[lane * (VM / G) + k] = A[k];
  __syncwarp(gm);
  C L[NA];
  constexpr MomentTable<M> MT = Moments<M>::T;
#pragma unroll
  for (int k = 0; k < NA; ++k) L[k] = sm[MT.idx[k]];
  __syncwarp(gm);
  C tr = 0;
#pragma unroll
  for (int r = 0; r < M; ++r) tr += L[pk(r, r)];
  C invd[M], pmin, pmax;
  const bool ok = (cnt >= M) && cholesky<M, C>(L, invd, sp.piv_tol_rel * tr, pmin, pmax);
  const C cond = (pmax / pmin) * (pmax / pmin);
  C *Ls = sm + StSmem<M, G>::SCR;
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < NA; ++k) Ls[k] = L[k];
  }
  __syncwarp(gm);
  if (!ok || (QUEUE && !(cond <= sp.cond_max))) {
    // deficient (decided in this precision unless queued) -> zeros
    if (QUEUE && cnt >= M) {
      *result = 2;
      return;
    }
    for (long long e = b + lane; e < e1; e += G) st4(coef + e, mk4<TS>(0, 0, 0, 0));
    *result = 1;
    *cond_out = INFINITY;
    return;
  }
  // entries of this lane, and how many of them the cache holds
  const int nloc = e1 > b + lane ? (int)((e1 - b - lane + G - 1) / G) : 0;
  const int ncache = KC > 0 ? min(nloc, KC) : 0;
  // ---- solve: lane k of the group solves right-hand side k (a warp issues one
  // solve for all of its groups' lanes at once instead of NR in a row; lanes
  // k >= NR repeat one) and the group reads the solutions back from shared memory
  static_assert(G >= NR, "one lane per right-hand side");
  const int kq = lane % NR;
  C lam[NR][M];
  {
    C bb[M], x[M];
#pragma unroll
    for (int r = 0; r < M; ++r) bb[r] = rhs<M, C>(kq, r);
    chol_solve_s<M, C>(Ls, invd, bb, x);
    if (lane < NR) {
#pragma unroll
      for (int r = 0; r < M; ++r) sm[lane * M + r] = x[r];
    }
    __syncwarp(gm);
#pragma unroll
    for (int k = 0; k < NR; ++k)
#pragma unroll
      for (int r = 0; r < M; ++r) lam[k][r] = sm[k * M + r];
    __syncwarp(gm);
  }
  // The Laplacian's refinement correction is kept apart (lamlo) instead of
  // being added into lam: its solution has entries ~100x its coefficients on
  // one-sided (free-surface, wall) rows, and rounding lam + d to FP32 would put
  // back an error A * (rounding of lam) into the moment conditions, which the
  // applied Laplacian sees divided by h.  Its coefficients are evaluated as
  // w (p.lam + p.lamlo).
  constexpr int KL = NR - 1;
  C lamlo[M];
#pragma unroll
  for (int r = 0; r < M; ++r) lamlo[r] = C(0);
  if constexpr (REFINE) {
    // residual b - sum_j c_j p_j of the coefficients as they will be stored
    C R[VR];
#pragma unroll
    for (int k = 0; k < VR; ++k) R[k] = C(0);
    for (int q = 0; q < ncache; ++q) {
      const float4 c4 = qw[q * G + lane];
      C p[M];
      basis_from_q<M, C>(c4, p);
      const C w = c4.w;
#pragma unroll
      for (int k = 0; k < NR; ++k) {
        C s = lam[k][0];   // p_0 = 1
#pragma unroll
        for (int r = 1; r < M; ++r) s = fma(p[r], lam[k][r], s);
        const C c = w * s;
        R[k * M] += c;
#pragma unroll
        for (int r = 1; r < M; ++r) R[k * M + r] = fma(c, p[r], R[k * M + r]);
      }
    }
    for (long long e0 = b + lane + (long long)ncache * G; e0 < e1; e0 += kGatherR * G) {
      V xs[kGatherR];
      bool oks[kGatherR];
      gather_row<kGatherR, G>(e0, e1, i, mi, col, pos, model, xs, oks);
#pragma unroll
      for (int u = 0; u < kGatherR; ++u) {
        C p[M];
        C w = basis_at<M, C>(xi, xs[u], hinv, t1, t2, sp, p);
        w = oks[u] ? w : C(0);
#pragma unroll
        for (int k = 0; k < NR; ++k) {
          C s = lam[k][0];   // p_0 = 1
#pragma unroll
          for (int r = 1; r < M; ++r) s = fma(p[r], lam[k][r], s);
          const C c = w * s;
          R[k * M] += c;
#pragma unroll
          for (int r = 1; r < M; ++r) R[k * M + r] = fma(c, p[r], R[k * M + r]);
        }
      }
    }
    reduce_scatter<G, VR>(R);
#pragma unroll
    for (int k = 0; k < VR / G; ++k) sm[lane * (VR / G) + k] = R[k];
    __syncwarp(gm);
    {
      // the corrections, one right-hand side per lane as above
      C rr[M], d[M];
#pragma unroll
      for (int r = 0; r < M; ++r) rr[r] = rhs<M, C>(kq, r) - sm[kq * M + r];
      __syncwarp(gm);   // every lane has its residual before the corrections overwrite it
      chol_solve_s<M, C>(Ls, invd, rr, d);
      if (lane < NR) {
#pragma unroll
        for (int r = 0; r < M; ++r) sm[lane * M + r] = d[r];
      }
      __syncwarp(gm);
#pragma unroll
      for (int k = 0; k < NR; ++k)
#pragma unroll
        for (int r = 0; r < M; ++r) {
          if (k == KL) lamlo[r] = sm[k * M + r];
          else lam[k][r] += sm[k * M + r];
        }
    }
    __syncwarp(gm);
  }
  // ---- coefficients
  const C h2inv = hinv * hinv;
  // the output record of one entry: w p.lambda_k (+ w p.lamlo for the
  // Laplacian) with the operator's scale 1/h or 1/h^2 folded into w
  auto coef_of = [&](const C (&p)[M], C w) -> vec4_t<TS> {
    const C wg = w * hinv, wl = w * h2inv;
    C s[NR];
#pragma unroll
    for (int k = 0; k < NR; ++k) {
      C v = lam[k][0];   // p_0 = 1
#pragma unroll
      for (int r = 1; r < M; ++r) v = fma(p[r], lam[k][r], v);
      if (REFINE && k == KL) {
        C sl = lamlo[0];
#pragma unroll
        for (int r = 1; r < M; ++r) sl = fma(p[r], lamlo[r], sl);
        v += sl;
      }
      s[k] = v;
    }
    if constexpr (M == 10) {
      return mk4<TS>(TS(wg * s[0]), TS(wg * s[1]), TS(wg * s[2]), TS(wl * s[3]));
    } else {
      const C gx = wg * fma(s[0], t1[0], s[1] * t2[0]);
      const C gy = wg * fma(s[0], t1[1], s[1] * t2[1]);
      const C gz = wg * fma(s[0], t1[2], s[1] * t2[2]);
      return mk4<TS>(TS(gx), TS(gy), TS(gz), TS(wl * s[2]));
    }
  };
  auto write_coef = [&](long long e, const C (&p)[M], C w) { st4(coef + e, coef_of(p, w)); };
  for (int q = 0; q < ncache; ++q) {
    const float4 c4 = qw[q * G + lane];
    C p[M];
    basis_from_q<M, C>(c4, p);
    if (c4.w != 0.f) write_coef(b + lane + (long long)q * G, p, C(c4.w));
    else st4(coef + b + lane + (long long)q * G, mk4<TS>(0, 0, 0, 0));
  }
  for (long long e0 = b + lane + (long long)ncache * G; e0 < e1; e0 += kGatherU<M> * G) {
    V xs[kGatherU<M>];
    bool oks[kGatherU<M>];
    gather_row<kGatherU<M>, G>(e0, e1, i, mi, col, pos, model, xs, oks);
#pragma unroll
    for (int u = 0; u < kGatherU<M>; ++u) {
    const long long e = e0 + (long long)u * G;
    if (e >= e1) break;
    vec4_t<TS> out = mk4<TS>(0, 0, 0, 0);
    if (oks[u]) {
      C p[M];
      const C w = basis_at<M, C>(xi, xs[u], hinv, t1, t2, sp, p);
      out = coef_of(p, w);
    }
    st4(coef + e, out);
    }
  }
  *result = 0;
  *cond_out = (float)cond;
}

// Main kernel: every particle of model (M == 10 ? 3D : 2D).
template <typename TS, typename C, int M, int G, bool REFINE, bool QUEUE>
__global__ void __launch_bounds__(kStThreads, sizeof(C) == 4 ? (M == 10 ? 4 : 6) : 1) k_stencil(
    int64_t n, const vec4_t<TS> *pos, const uint8_t *model, const vec4_t<TS> *frame,
    const long long *row_ptr, const int32_t *col, vec4_t<TS> *coef, uint8_t *status,
    float *cond, StParams<C> sp, DevStatus *st, int32_t *queue) {
  constexpr int NA = Basis<M>::NA, NR = Basis<M>::NR;
  constexpr int SMG = StSmem<M, G>::PER_GROUP;
  constexpr int KC = StCache<C, M, G>::KC;
  extern __shared__ __align__(16) unsigned char st_smem[];
  float4 *qcache = reinterpret_cast<float4 *>(st_smem);
  C *smem = reinterpret_cast<C *>(st_smem + StCache<C, M, G>::BYTES);
  const int grp = threadIdx.x / G;
  C *sm = smem + grp * SMG;
  float4 *qw = qcache + grp * KC * G;
  const int lane = threadIdx.x & (G - 1);
  const int64_t gid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / G;
  const int64_t ngroups = ((int64_t)gridDim.x * blockDim.x) / G;
  const uint8_t want = M == 10 ? MAFP_MODEL_3D : MAFP_MODEL_2D;
  for (int64_t i = gid; i < n; i += ngroups) {
    if (model[i] != want) continue;   // uniform within the group
    int res;
    float cd = 0.0f;
    stencil_particle<TS, C, M, G, REFINE, QUEUE, KC>(i, pos, model, frame, row_ptr, col, coef,
                                                     sp, sm, &res, &cd, qw);
    if (lane == 0) {
      if (res == 2) {
        const int slot = atomicAdd(&st->fallback_count, 1);
        queue[slot] = (int32_t)i;
      } else {
        status[i] = res == 0 ? MAFP_STENCIL_OK : MAFP_STENCIL_DEFICIENT;
        cond[i] = res == 0 ? cd : INFINITY;
        if (res == 1) inc_ll(&st->n_deficient);
      }
    }
  }
}

// FP64 redo of the queued particles of one model (FP32 storage).
template <int M, int G>
__global__ void __launch_bounds__(kStThreads) k_stencil_redo(
    const float4 *pos, const uint8_t *model, const float4 *frame, const long long *row_ptr,
    const int32_t *col, float4 *coef, uint8_t *status, float *cond, StParams<double> sp,
    DevStatus *st, const int32_t *queue) {
  constexpr int NA = Basis<M>::NA, NR = Basis<M>::NR;
  constexpr int SMG = StSmem<M, G>::PER_GROUP;
  __shared__ double smem[(kStThreads / G) * SMG];
  const int grp = threadIdx.x / G;
  double *sm = smem + grp * SMG;
  const int lane = threadIdx.x & (G - 1);
  const int64_t gid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / G;
  const int64_t ngroups = ((int64_t)gridDim.x * blockDim.x) / G;
  const int nq = st->fallback_count;
  const uint8_t want = M == 10 ? MAFP_MODEL_3D : MAFP_MODEL_2D;
  for (int64_t q = gid; q < nq; q += ngroups) {
    const int64_t i = queue[q];
    if (model[i] != want) continue;
    int res;
    float cd = 0.0f;
    stencil_particle<float, double, M, G, false, false>(i, pos, model, frame, row_ptr, col, coef,
                                                         sp, sm, &res, &cd);
    if (lane == 0) {
      status[i] = res == 0 ? MAFP_STENCIL_FP64 : MAFP_STENCIL_DEFICIENT;
      cond[i] = res == 0 ? cd : INFINITY;
      if (res == 1) inc_ll(&st->n_deficient);
      else inc_ll(&st->n_fp64_stencil);
    }
  }
}


template <typename TS, typename C, int M, int G, bool REFINE, bool QUEUE>
static void launch_stencil(mafp_ctx *ctx, cudaStream_t s, int64_t n, const void *pos_h,
                           const uint8_t *model, const void *frame, const long long *rp,
                           const int32_t *col, void *coef, uint8_t *status, float *cond,
                           const StParams<C> &sp) {
  using V = vec4_t<TS>;
  static const KernelName name("k_stencil<%s,M=%d,G=%d,%s>", sizeof(TS) == 4 ? "f32" : "f64",
                               M, G, REFINE ? "refined" : "plain");
  const int blocks = grid_for(n * G, kStThreads, sm_count() * 64);
  constexpr int smem = StCache<C, M, G>::SMEM;
  // the dynamic shared-memory limit is a per-device setting of the function
  static unsigned long long attr_devices = 0;
  if (smem > 48 * 1024 && first_on_device(&attr_devices, ctx->device))
    cudaFuncSetAttribute(k_stencil<TS, C, M, G, REFINE, QUEUE>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  MAFP_TIMED(ctx, s, name.s,
             k_stencil<TS, C, M, G, REFINE, QUEUE><<<blocks, kStThreads, smem, s>>>(
                 n, (const V *)pos_h, model, (const V *)frame, rp, col, (V *)coef, status, cond,
                 sp, ctx->d_status, ctx->fallback));
}

// Group size G chosen at run time (tuning), instantiated for 8/16/32 (3D) and 4/8/16 (2D).
template <typename TS, typename C, bool REFINE, bool QUEUE>
static int dispatch_stencils(mafp_ctx *ctx, cudaStream_t s, int64_t n, const void *pos_h,
                             const uint8_t *model, const void *frame, const long long *rp,
                             const int32_t *col, void *coef, uint8_t *status, float *cond,
                             const StParams<C> &sp) {
  switch (ctx->tune.stencil3d_group) {
    case 8: launch_stencil<TS, C, 10, 8, REFINE, QUEUE>(ctx, s, n, pos_h, model, frame, rp, col, coef, status, cond, sp); break;
    case 16: launch_stencil<TS, C, 10, 16, REFINE, QUEUE>(ctx, s, n, pos_h, model, frame, rp, col, coef, status, cond, sp); break;
    default: launch_stencil<TS, C, 10, 32, REFINE, QUEUE>(ctx, s, n, pos_h, model, frame, rp, col, coef, status, cond, sp); break;
  }
  switch (ctx->tune.stencil2d_group) {
    case 4: launch_stencil<TS, C, 6, 4, REFINE, QUEUE>(ctx, s, n, pos_h, model, frame, rp, col, coef, status, cond, sp); break;
    case 16: launch_stencil<TS, C, 6, 16, REFINE, QUEUE>(ctx, s, n, pos_h, model, frame, rp, col, coef, status, cond, sp); break;
    default: launch_stencil<TS, C, 6, 8, REFINE, QUEUE>(ctx, s, n, pos_h, model, frame, rp, col, coef, status, cond, sp); break;
  }
  MAFP_LAUNCH_CHECK(ctx);
  return MAFP_OK;
}

int build_stencils(mafp_ctx *ctx, int64_t n, int32_t dtype, const void *pos_h,
                   const uint8_t *model, const void *frame, const int64_t *row_ptr,
                   const int32_t *col, void *coef, uint8_t *status, float *cond, cudaStream_t s) {
  const long long *rp = reinterpret_cast<const long long *>(row_ptr);
  const int sms = sm_count();
  if (dtype == MAFP_F64) {
    const StParams<double> sp = make_params<double>(ctx->prm, 1e-12);
    return dispatch_stencils<double, double, false, false>(ctx, s, n, pos_h, model, frame, rp,
                                                          col, coef, status, cond, sp);
  }
  const StParams<float> sp = make_params<float>(ctx->prm, 1e-6);
  const StParams<double> sp64 = make_params<double>(ctx->prm, 1e-12);
  MAFP_TIMED(ctx, s, "k_reset_queue", k_reset_queue<<<1, 1, 0, s>>>(ctx->d_status));
  int rc = dtype == MAFP_F32_PLAIN
               ? dispatch_stencils<float, float, false, true>(ctx, s, n, pos_h, model, frame, rp,
                                                             col, coef, status, cond, sp)
               : dispatch_stencils<float, float, true, true>(ctx, s, n, pos_h, model, frame, rp,
                                                            col, coef, status, cond, sp);
  if (rc) return rc;
  // FP64 redo: small groups keep the per-particle factorisation, repeated in
  // every lane of a group, from dominating the slow FP64 pipe
  MAFP_TIMED(ctx, s, "k_stencil_redo<10,4>",
             k_stencil_redo<10, 4><<<sms * 32, kStThreads, 0, s>>>(
      (const float4 *)pos_h, model, (const float4 *)frame, rp, col, (float4 *)coef, status, cond,
      sp64, ctx->d_status, ctx->fallback));
  MAFP_TIMED(ctx, s, "k_stencil_redo<6,4>",
             k_stencil_redo<6, 4><<<sms * 32, kStThreads, 0, s>>>(
      (const float4 *)pos_h, model, (const float4 *)frame, rp, col, (float4 *)coef, status, cond,
      sp64, ctx->d_status, ctx->fallback));
  MAFP_LAUNCH_CHECK(ctx);
  return MAFP_OK;
}

}  // namespace mafp
