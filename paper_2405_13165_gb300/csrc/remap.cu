// remap.cu -- model transition with data mapping (Sec. 5, Algs. 3 and 4).
//  1. owner: every interior / free-surface 3D particle b that neighbours a
//     particle flagged 3D -> 2D finds its nearest 3D wall particle j^w in S_b
//     (squared distance in FP64, ties to the lower index); b is deleted and
//     mapped onto j^w when j^w is flagged.  The candidates b are marked from
//     the rows of the flagged particles (S is symmetric), so only they search.
//     gamma of every 2D -> 3D particle.
//  2. scans: survivor positions, appended-particle offsets, n_out.
//  3. survivors copied; 3D -> 2D particles aggregate their set T_i;
//     2D -> 3D particles split their mass and emit gamma new particles.
#include "internal.cuh"
#include "state.cuh"

namespace mafp {

__device__ __forceinline__ double dist2_64(double xi, double yi, double zi, double xj, double yj,
                                           double zj) {
  const double dx = __dsub_rn(xj, xi), dy = __dsub_rn(yj, yi), dz = __dsub_rn(zj, zi);
  return __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
}

// gamma = ceil(H / (c_psi h3D)) in FP64 (Sec. 5.2), 0 when H <= 0.
__device__ __forceinline__ int gamma_of(double H, double h3d, double c_psi) {
  if (!(H > 0.0)) return 0;
  const double psi_t = __dmul_rn(c_psi, h3d);
  return (int)ceil(__ddiv_rn(H, psi_t));
}

// Every particle: no owner yet, kept, and gamma of the 2D -> 3D particles.
template <typename T>
__global__ void k_owner_seed(int64_t n, StateT<T> in, const uint8_t *flag, int32_t *owner,
                             int32_t *keep, int32_t *gam, double c_psi) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b < n; b += stride) {
    owner[b] = -1;
    keep[b] = 1;
    gam[b] = (flag[b] == 2 && in.model[b] == MAFP_MODEL_2D)
                 ? gamma_of((double)in.hfilm[b], (double)in.h3d[b], c_psi)
                 : 0;
  }
}

// Candidates of Alg. 3: the interior / free-surface 3D particles b that have a
// 3D particle j flagged 3D -> 2D in S_b.  S is symmetric (Eq. Nbd), so one
// warp per flagged j marks the candidates in its own row (owner[b] = -2);
// only they search for a wall below.
__global__ void k_owner_mark(int64_t n, const uint8_t *model, const uint8_t *type,
                             const uint8_t *flag, const long long *row_ptr, const int32_t *col,
                             int32_t *owner) {
  const int lane = threadIdx.x & 31;
  const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  // the warp tests 32 particles at once and walks the rows of the flagged ones
  for (int64_t j0 = wid * 32; j0 < n; j0 += nwarps * 32) {
    const int64_t jl = j0 + lane;
    unsigned m = __ballot_sync(0xffffffffu,
                               jl < n && flag[jl] == 1 && model[jl] == MAFP_MODEL_3D);
    while (m) {
      const int64_t j = j0 + __ffs(m) - 1;
      m &= m - 1;
      const long long r0 = row_ptr[j], r1 = row_ptr[j + 1];
      for (long long e = r0 + lane; e < r1; e += 32) {
        const int b = col[e];
        if (model[b] == MAFP_MODEL_3D && type[b] != MAFP_TYPE_WALL) owner[b] = -2;
      }
    }
  }
}

// Every candidate b finds its nearest 3D wall particle j^w in S_b (FP64 squared
// distance, ties to the lower index) and is mapped onto it when j^w is flagged.
template <typename T>
__global__ void k_owner(int64_t n, StateT<T> in, const uint8_t *flag, const long long *row_ptr,
                        const int32_t *col, int32_t *owner, int32_t *keep) {
  const int lane = threadIdx.x & 31;
  const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  // the warp tests 32 particles at once and searches for the marked ones
  for (int64_t b0 = wid * 32; b0 < n; b0 += nwarps * 32) {
    const int64_t bl = b0 + lane;
    unsigned mk = __ballot_sync(0xffffffffu, bl < n && owner[bl] == -2);
    while (mk) {
      const int64_t b = b0 + __ffs(mk) - 1;
      mk &= mk - 1;
      const long long r0 = row_ptr[b], r1 = row_ptr[b + 1];
      const vec4_t<T> xb = ld4(in.pos_h + b);
      double best = INFINITY;
      int jw = INT_MAX;
      for (long long e = r0 + lane; e < r1; e += 32) {
        const int j = col[e];
        if (in.model[j] != MAFP_MODEL_3D || in.type[j] != MAFP_TYPE_WALL) continue;
        const vec4_t<T> xj = ld4(in.pos_h + j);
        const double d2 = dist2_64(xb.x, xb.y, xb.z, xj.x, xj.y, xj.z);
        if (d2 < best || (d2 == best && j < jw)) {
          best = d2;
          jw = j;
        }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const double ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int oj = __shfl_xor_sync(0xffffffffu, jw, o);
        if (ob < best || (ob == best && oj < jw)) {
          best = ob;
          jw = oj;
        }
      }
      const int32_t own = (jw != INT_MAX && flag[jw] == 1) ? jw : -1;
      if (lane == 0) {
        owner[b] = own;
        keep[b] = own < 0 ? 1 : 0;
      }
    }
  }
}

__global__ void k_remap_count(const long long *keep_scan, const long long *gam_scan, int64_t n,
                              long long cap_out, int64_t *n_out_dev, DevStatus *st) {
  const long long n_out = keep_scan[n] + gam_scan[n];
  st->n_out = n_out;
  if (n_out_dev) *n_out_dev = n_out;
  st->remap_scratch[0] = n_out > cap_out ? 1 : 0;
  if (n_out > cap_out) set_error(st, MAFP_ECAPACITY, n_out);
}

template <typename T>
__device__ __forceinline__ T droplet_diameter(double m, double rho) {
  return (T)cbrt(6.0 * m / (3.141592653589793 * rho));
}

// Survivors: copy, then the 2D -> 3D particle's own update (Alg. 4 data mapping).
template <typename T>
__global__ void k_survivors(int64_t n, StateT<T> in, StateT<T> out, const uint8_t *flag,
                            const int32_t *owner, const long long *keep_scan,
                            const int32_t *gam, int32_t *old2new, const DevStatus *st) {
  const bool skip = st->remap_scratch[0] != 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    if (owner[i] >= 0) {
      old2new[i] = -1;
      continue;
    }
    const long long o = keep_scan[i];
    old2new[i] = (int32_t)o;
    if (skip) continue;
    vec4_t<T> p = ld4(in.pos_h + i);
    st4(out.vp + o, ld4(in.vp + i));
    st4(out.normal + o, ld4(in.normal + i));
    out.rho[o] = in.rho[i];
    out.eta[o] = in.eta[i];
    out.mass[o] = in.mass[i];
    out.diam[o] = in.diam[i];
    out.hfilm[o] = in.hfilm[i];
    out.h3d[o] = in.h3d[i];
    out.model[o] = in.model[i];
    out.type[o] = in.type[i];
    out.last[o] = 0;
    if (flag[i] == 2 && in.model[i] == MAFP_MODEL_2D) {
      const int g = gam[i];
      const double m = (double)in.mass[i] / (1.0 + (double)g);
      out.mass[o] = (T)m;
      out.diam[o] = droplet_diameter<T>(m, (double)in.rho[i]);
      p.w = in.h3d[i];
      out.hfilm[o] = T(0);
      out.model[o] = MAFP_MODEL_3D;
      out.type[o] = MAFP_TYPE_WALL;
      out.last[o] = 1;
    }
    st4(out.pos_h + o, p);
  }
}

// 3D -> 2D data mapping of Sec. 5.1 for each flagged particle (one warp each).
template <typename T>
__global__ void k_to2d(int64_t n, StateT<T> in, StateT<T> out, const uint8_t *flag,
                       const int32_t *owner, const long long *keep_scan,
                       const long long *row_ptr, const int32_t *col, const DevStatus *st) {
  if (st->remap_scratch[0] != 0) return;
  const int lane = threadIdx.x & 31;
  const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  // the warp tests 32 particles at once and maps the flagged ones
  for (int64_t i0 = wid * 32; i0 < n; i0 += nwarps * 32) {
    const int64_t il = i0 + lane;
    unsigned fl = __ballot_sync(0xffffffffu,
                                il < n && flag[il] == 1 && in.model[il] == MAFP_MODEL_3D);
    while (fl) {
      const int64_t i = i0 + __ffs(fl) - 1;
      fl &= fl - 1;
      const vec4_t<T> xi = ld4(in.pos_h + i), ni = ld4(in.normal + i);
      T s[7] = {0, 0, 0, 0, 0, 0, 0};  // vp(4), rho, eta, mass
      T H = 0;
      int cnt = 0;
      for (long long e = row_ptr[i] + lane; e < row_ptr[i + 1]; e += 32) {
        const int b = col[e];
        if (owner[b] != (int32_t)i) continue;
        const vec4_t<T> v = ld4(in.vp + b), xb = ld4(in.pos_h + b);
        s[0] += v.x; s[1] += v.y; s[2] += v.z; s[3] += v.w;
        s[4] += in.rho[b];
        s[5] += in.eta[b];
        s[6] += in.mass[b];
        const T dn = fabs((xb.x - xi.x) * ni.x + (xb.y - xi.y) * ni.y + (xb.z - xi.z) * ni.z);
        H = dn > H ? dn : H;
        ++cnt;
      }
#pragma unroll
      for (int k = 0; k < 7; ++k) s[k] = group_sum<32>(s[k]);
      cnt = group_sum<32>(cnt);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const T oh = __shfl_xor_sync(0xffffffffu, H, o);
        H = oh > H ? oh : H;
      }
      if (lane == 0) {
        const long long o = keep_scan[i];
        const vec4_t<T> v = ld4(in.vp + i);
        const T k = T(1) + T(cnt);
        st4(out.vp + o, mk4<T>((v.x + s[0]) / k, (v.y + s[1]) / k, (v.z + s[2]) / k, (v.w + s[3]) / k));
        const T rho = (in.rho[i] + s[4]) / k;
        const T m = in.mass[i] + s[6];
        out.rho[o] = rho;
        out.eta[o] = (in.eta[i] + s[5]) / k;
        out.mass[o] = m;
        out.diam[o] = droplet_diameter<T>((double)m, (double)rho);
        out.hfilm[o] = H;
        out.model[o] = MAFP_MODEL_2D;
        out.type[o] = MAFP_TYPE_WALL;
        out.last[o] = 1;
      }
    }
  }
}

// Alg. 4 particle addition: x_i + (k psi) n_i, k = 1..gamma, psi = H / gamma.
template <typename T>
__global__ void k_append(int64_t n, StateT<T> in, StateT<T> out, const int32_t *gam,
                         const long long *keep_scan, const long long *gam_scan,
                         const DevStatus *st) {
  if (st->remap_scratch[0] != 0) return;
  const long long n_keep = keep_scan[n];
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int g = gam[i];
    if (g == 0) continue;
    const vec4_t<T> x = ld4(in.pos_h + i), nn = ld4(in.normal + i), v = ld4(in.vp + i);
    const double H = (double)in.hfilm[i];
    const double psi = __ddiv_rn(H, (double)g);
    const double m = (double)in.mass[i] / (1.0 + (double)g);
    const T diam = droplet_diameter<T>(m, (double)in.rho[i]);
    const long long base = n_keep + gam_scan[i];
    for (int k = 1; k <= g; ++k) {
      const long long o = base + k - 1;
      const double kp = __dmul_rn((double)k, psi);
      st4(out.pos_h + o, mk4<T>((T)__dadd_rn((double)x.x, __dmul_rn(kp, (double)nn.x)),
                                (T)__dadd_rn((double)x.y, __dmul_rn(kp, (double)nn.y)),
                                (T)__dadd_rn((double)x.z, __dmul_rn(kp, (double)nn.z)),
                                in.h3d[i]));
      st4(out.vp + o, v);
      st4(out.normal + o, nn);
      out.rho[o] = in.rho[i];
      out.eta[o] = in.eta[i];
      out.mass[o] = (T)m;
      out.diam[o] = diam;
      out.hfilm[o] = T(0);
      out.h3d[o] = in.h3d[i];
      out.model[o] = MAFP_MODEL_3D;
      out.type[o] = k == g ? MAFP_TYPE_FREE_SURFACE : MAFP_TYPE_INTERIOR;
      out.last[o] = 1;
    }
  }
}

template <typename T>
static int remap_t(mafp_ctx *ctx, int64_t n, const mafp_state *in_, const uint8_t *flag,
                   const long long *rp, const int32_t *col, const mafp_state *out_,
                   int64_t cap_out, int32_t *old2new, int64_t *n_out_dev, cudaStream_t s) {
  StateT<T> in = cast_state<T>(in_), out = cast_state<T>(out_);
  int32_t *owner = ctx->remap_i32, *keep = ctx->remap_i32 + n, *gam = ctx->remap_i32 + 2 * n;
  long long *keep_scan = reinterpret_cast<long long *>(ctx->remap_i64);
  long long *gam_scan = keep_scan + (n + 1);
  const int sms = sm_count();
  MAFP_TIMED(ctx, s, "k_owner_seed<T>",
             k_owner_seed<T><<<grid_for(n, 256, sms * 16), 256, 0, s>>>(n, in, flag, owner, keep,
                                                                    gam, ctx->prm.c_psi));
  MAFP_TIMED(ctx, s, "k_owner_mark",
             k_owner_mark<<<grid_for(n * 32, 256, sms * 32), 256, 0, s>>>(n, in.model, in.type, flag,
                                                                       rp, col, owner));
  MAFP_TIMED(ctx, s, "k_owner<T>",
             k_owner<T><<<grid_for(n * 32, 256, sms * 32), 256, 0, s>>>(n, in, flag, rp, col, owner,
                                                                     keep));
  MAFP_LAUNCH_CHECK(ctx);
  int rc = scan_i32_to_i64(ctx, keep, keep_scan, n, s);
  if (rc) return rc;
  rc = scan_i32_to_i64(ctx, gam, gam_scan, n, s);
  if (rc) return rc;
  MAFP_TIMED(ctx, s, "k_remap_count",
             k_remap_count<<<1, 1, 0, s>>>(keep_scan, gam_scan, n, cap_out, n_out_dev, ctx->d_status));
  MAFP_TIMED(ctx, s, "k_survivors<T>",
             k_survivors<T><<<grid_for(n, 256, sms * 16), 256, 0, s>>>(n, in, out, flag, owner, keep_scan,
                                                             gam, old2new, ctx->d_status));
  MAFP_TIMED(ctx, s, "k_to2d<T>",
             k_to2d<T><<<grid_for(n * 32, 256, sms * 32), 256, 0, s>>>(n, in, out, flag, owner, keep_scan,
                                                             rp, col, ctx->d_status));
  MAFP_TIMED(ctx, s, "k_append<T>",
             k_append<T><<<grid_for(n, 256, sms * 16), 256, 0, s>>>(n, in, out, gam, keep_scan, gam_scan,
                                                          ctx->d_status));
  MAFP_LAUNCH_CHECK(ctx);
  return MAFP_OK;
}

int remap_switched(mafp_ctx *ctx, int64_t n, int32_t dtype, const mafp_state *in,
                   const uint8_t *flag, const int64_t *row_ptr, const int32_t *col,
                   const mafp_state *out, int64_t cap_out, int32_t *old2new, int64_t *n_out_dev,
                   cudaStream_t s) {
  const long long *rp = reinterpret_cast<const long long *>(row_ptr);
  if (dtype == MAFP_F64)
    return remap_t<double>(ctx, n, in, flag, rp, col, out, cap_out, old2new, n_out_dev, s);
  return remap_t<float>(ctx, n, in, flag, rp, col, out, cap_out, old2new, n_out_dev, s);
}

}  // namespace mafp
