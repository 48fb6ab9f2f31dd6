// apply.cu -- stencil application of Eq. GFDM_Definition as a ragged gather-SpMV
// (four fields x four operators per row) and its transpose, either gathered
// through the symmetric-structure map (deterministic) or scattered with
// atomic adds (no map needed).
#include "internal.cuh"

namespace mafp {

constexpr int kApThreads = 256;

// out[i][f][op] = sum_{e in row i} coef[e].op * (fields[col[e]].f - fields[i].f)
// The stencils reproduce constants (sum_j c_ij = 0, order-2 consistency of
// Sec. 2.3), so this is Eq. GFDM_Definition; differencing first removes the
// u_i * sum_j c_ij term that FP32 rounding of the coefficients leaves behind.
// A group of G lanes per row; lanes stride over the row with U loads in flight.
template <typename T, int G, int U>
__global__ void __launch_bounds__(kApThreads) k_apply(int64_t n, const long long *row_ptr,
                                                      const int32_t *col,
                                                      const vec4_t<T> *coef,
                                                      const vec4_t<T> *fields, T *out) {
  using V = vec4_t<T>;
  const int lane = threadIdx.x & (G - 1);
  const int64_t gid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / G;
  const int64_t ngroups = ((int64_t)gridDim.x * blockDim.x) / G;
  for (int64_t i = gid; i < n; i += ngroups) {
    const long long b = row_ptr[i], e1 = row_ptr[i + 1];
    const V fi = ld4(fields + i);
    T acc[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) acc[k] = T(0);
    // U entries per lane in flight; past the row end the slot reads particle
    // i itself with a zero coefficient (an exact zero contribution)
    for (long long e = b + lane; e < e1; e += U * G) {
      int j[U];
      V c[U], f[U];
#pragma unroll
      for (int u = 0; u < U; ++u) j[u] = e + u * G < e1 ? __ldg(col + e + u * G) : (int)i;
#pragma unroll
      for (int u = 0; u < U; ++u) c[u] = e + u * G < e1 ? ld4(coef + e + u * G) : mk4<T>(0, 0, 0, 0);
#pragma unroll
      for (int u = 0; u < U; ++u) f[u] = ld4(fields + j[u]);
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const T fv[4] = {f[u].x - fi.x, f[u].y - fi.y, f[u].z - fi.z, f[u].w - fi.w};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          acc[4 * q + 0] += c[u].x * fv[q];
          acc[4 * q + 1] += c[u].y * fv[q];
          acc[4 * q + 2] += c[u].z * fv[q];
          acc[4 * q + 3] += c[u].w * fv[q];
        }
      }
    }
    reduce_scatter<G, 16>(acc);
    constexpr int PER = 16 / G;
    T *o = out + 16 * i + lane * PER;
    if constexpr (PER == 2) {
      if constexpr (sizeof(T) == 4) {
        *reinterpret_cast<float2 *>(o) = make_float2(acc[0], acc[1]);
      } else {
        *reinterpret_cast<double2 *>(o) = make_double2(acc[0], acc[1]);
      }
    } else if constexpr (PER == 4) {
      st4(reinterpret_cast<V *>(o), mk4<T>(acc[0], acc[1], acc[2], acc[3]));
    } else {
#pragma unroll
      for (int k = 0; k < PER; ++k) o[k] = acc[k];
    }
  }
}

// Exact adjoint of k_apply with respect to the fields:
// gfields[j][f] = sum_{e in row j} sum_op (coef[(i, j)].op gout[i][f][op] - coef[e].op gout[j][f][op]),
// i = col[e], (i, j) found at row_ptr[i] + tloc[e]; the second term is the
// adjoint of the -u_j sum_k c_jk part of the differenced form.
template <typename T, int G>
__global__ void __launch_bounds__(kApThreads) k_apply_T(int64_t n, const long long *row_ptr,
                                                        const int32_t *col,
                                                        const uint16_t *tloc,
                                                        const vec4_t<T> *coef,
                                                        const vec4_t<T> *gout,
                                                        vec4_t<T> *gfields) {
  using V = vec4_t<T>;
  const int lane = threadIdx.x & (G - 1);
  const int64_t gid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / G;
  const int64_t ngroups = ((int64_t)gridDim.x * blockDim.x) / G;
  for (int64_t jr = gid; jr < n; jr += ngroups) {
    const long long b = row_ptr[jr], e1 = row_ptr[jr + 1];
    T acc[G < 4 ? 4 : G];
#pragma unroll
    for (int k = 0; k < (G < 4 ? 4 : G); ++k) acc[k] = T(0);
    V csum = mk4<T>(0, 0, 0, 0);
    for (long long e = b + lane; e < e1; e += G) {
      const int i = __ldg(col + e);
      const long long ei = row_ptr[i] + tloc[e];
      const V c = ld4(coef + ei);
      const V cs = ld4(coef + e);
      csum.x += cs.x; csum.y += cs.y; csum.z += cs.z; csum.w += cs.w;
#pragma unroll
      for (int f = 0; f < 4; ++f) {
        const V g = ld4(gout + 4 * (int64_t)i + f);
        acc[f] += c.x * g.x + c.y * g.y + c.z * g.z + c.w * g.w;
      }
    }
#pragma unroll
    for (int f = 0; f < 4; ++f) {
      const V g = ld4(gout + 4 * jr + f);
      acc[f] -= csum.x * g.x + csum.y * g.y + csum.z * g.z + csum.w * g.w;
    }
    reduce_scatter<G, (G < 4 ? 4 : G)>(acc);
    T *o = reinterpret_cast<T *>(gfields + jr);
    if (lane < 4) o[lane] = acc[0];
  }
}

// The same adjoint scattered from the rows: row i adds coef[e] . gout[i][f] to
// gfields[col[e]] (one vector atomic per entry in FP32) and subtracts its own
// row sums once; needs no transpose map, sums in an unspecified order.
template <typename T>
__device__ __forceinline__ void add4(vec4_t<T> *p, T x, T y, T z, T w);
template <>
__device__ __forceinline__ void add4<float>(float4 *p, float x, float y, float z, float w) {
  atomicAdd(p, make_float4(x, y, z, w));
}
template <>
__device__ __forceinline__ void add4<double>(double4_16a *p, double x, double y, double z,
                                             double w) {
  double *q = reinterpret_cast<double *>(p);
  atomicAdd(q, x);
  atomicAdd(q + 1, y);
  atomicAdd(q + 2, z);
  atomicAdd(q + 3, w);
}

template <typename T, int G>
__global__ void __launch_bounds__(kApThreads) k_apply_T_scatter(int64_t n,
                                                                const long long *row_ptr,
                                                                const int32_t *col,
                                                                const vec4_t<T> *coef,
                                                                const vec4_t<T> *gout,
                                                                vec4_t<T> *gfields) {
  using V = vec4_t<T>;
  const int lane = threadIdx.x & (G - 1);
  const int64_t gid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / G;
  const int64_t ngroups = ((int64_t)gridDim.x * blockDim.x) / G;
  for (int64_t i = gid; i < n; i += ngroups) {
    const long long b = row_ptr[i], e1 = row_ptr[i + 1];
    V g[4];
#pragma unroll
    for (int f = 0; f < 4; ++f) g[f] = ld4(gout + 4 * i + f);
    T cs[4] = {0, 0, 0, 0};
    constexpr int U = 4;   // entries per lane with their loads in flight together
    for (long long e = b + lane; e < e1; e += U * G) {
      int j[U];
      V c[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const bool in = e + u * G < e1;
        j[u] = in ? __ldg(col + e + u * G) : -1;
        c[u] = in ? ld4(coef + e + u * G) : mk4<T>(0, 0, 0, 0);
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        if (j[u] < 0) break;
        cs[0] += c[u].x; cs[1] += c[u].y; cs[2] += c[u].z; cs[3] += c[u].w;
        T v[4];
#pragma unroll
        for (int f = 0; f < 4; ++f)
          v[f] = c[u].x * g[f].x + c[u].y * g[f].y + c[u].z * g[f].z + c[u].w * g[f].w;
        add4<T>(gfields + j[u], v[0], v[1], v[2], v[3]);
      }
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) cs[k] = group_sum<G>(cs[k]);
    if (lane == 0) {
      T v[4];
#pragma unroll
      for (int f = 0; f < 4; ++f)
        v[f] = -(cs[0] * g[f].x + cs[1] * g[f].y + cs[2] * g[f].z + cs[3] * g[f].w);
      add4<T>(gfields + i, v[0], v[1], v[2], v[3]);
    }
  }
}

template <typename T>
static void launch_apply(mafp_ctx *ctx, cudaStream_t s, int64_t n, const long long *rp,
                         const int32_t *col, const void *coef, const void *fields, void *out) {
  using V = vec4_t<T>;
  const int G = ctx->tune.apply_group;
  const int blocks = grid_for(n * G, kApThreads, sm_count() * 64);
  constexpr int U = sizeof(T) == 4 ? 8 : 2;
  const V *c = (const V *)coef, *f = (const V *)fields;
  T *o = (T *)out;
  if (G == 4) {
    MAFP_TIMED(ctx, s, "k_apply<G=4>", k_apply<T, 4, U><<<blocks, kApThreads, 0, s>>>(n, rp, col, c, f, o));
  } else if (G == 16) {
    MAFP_TIMED(ctx, s, "k_apply<G=16>", k_apply<T, 16, U><<<blocks, kApThreads, 0, s>>>(n, rp, col, c, f, o));
  } else {
    MAFP_TIMED(ctx, s, "k_apply<G=8>", k_apply<T, 8, U><<<blocks, kApThreads, 0, s>>>(n, rp, col, c, f, o));
  }
}

template <typename T>
static int launch_apply_T(mafp_ctx *ctx, cudaStream_t s, int64_t n, const long long *rp,
                           const int32_t *col, const uint16_t *tloc, const void *coef,
                           const void *gout, void *gfields) {
  using V = vec4_t<T>;
  const int G = ctx->tune.apply_group;
  const int blocks = grid_for(n * G, kApThreads, sm_count() * 64);
  const V *c = (const V *)coef, *g = (const V *)gout;
  V *o = (V *)gfields;
  if (!tloc) {
    MAFP_CUDA_TRY(ctx, cudaMemsetAsync(gfields, 0, (size_t)n * sizeof(V), s));
    if (G == 4) {
      MAFP_TIMED(ctx, s, "k_apply_T_scatter<G=4>", k_apply_T_scatter<T, 4><<<blocks, kApThreads, 0, s>>>(n, rp, col, c, g, o));
    } else if (G == 16) {
      MAFP_TIMED(ctx, s, "k_apply_T_scatter<G=16>", k_apply_T_scatter<T, 16><<<blocks, kApThreads, 0, s>>>(n, rp, col, c, g, o));
    } else {
      MAFP_TIMED(ctx, s, "k_apply_T_scatter<G=8>", k_apply_T_scatter<T, 8><<<blocks, kApThreads, 0, s>>>(n, rp, col, c, g, o));
    }
    return MAFP_OK;
  }
  if (G == 4) {
    MAFP_TIMED(ctx, s, "k_apply_T<G=4>", k_apply_T<T, 4><<<blocks, kApThreads, 0, s>>>(n, rp, col, tloc, c, g, o));
  } else if (G == 16) {
    MAFP_TIMED(ctx, s, "k_apply_T<G=16>", k_apply_T<T, 16><<<blocks, kApThreads, 0, s>>>(n, rp, col, tloc, c, g, o));
  } else {
    MAFP_TIMED(ctx, s, "k_apply_T<G=8>", k_apply_T<T, 8><<<blocks, kApThreads, 0, s>>>(n, rp, col, tloc, c, g, o));
  }
  return MAFP_OK;
}

int apply_ops(mafp_ctx *ctx, int64_t n, int32_t dtype, const int64_t *row_ptr, const int32_t *col,
              const void *coef, const void *fields, void *out, cudaStream_t s) {
  const long long *rp = reinterpret_cast<const long long *>(row_ptr);
  if (dtype == MAFP_F64) launch_apply<double>(ctx, s, n, rp, col, coef, fields, out);
  else launch_apply<float>(ctx, s, n, rp, col, coef, fields, out);
  MAFP_LAUNCH_CHECK(ctx);
  return MAFP_OK;
}

int apply_ops_backward(mafp_ctx *ctx, int64_t n, int32_t dtype, const int64_t *row_ptr,
                       const int32_t *col, const uint16_t *tloc, const void *coef,
                       const void *gout, void *gfields, cudaStream_t s) {
  const long long *rp = reinterpret_cast<const long long *>(row_ptr);
  const int rc = dtype == MAFP_F64
                     ? launch_apply_T<double>(ctx, s, n, rp, col, tloc, coef, gout, gfields)
                     : launch_apply_T<float>(ctx, s, n, rp, col, tloc, coef, gout, gfields);
  if (rc) return rc;
  MAFP_LAUNCH_CHECK(ctx);
  return MAFP_OK;
}

}  // namespace mafp
