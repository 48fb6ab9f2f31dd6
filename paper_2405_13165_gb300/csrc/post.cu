// post.cu -- film momentum update of the depth-averaged model (Eq. FilmMomentum)
// and the post-processing quantities of Sec. 7.3: fluid flux through a plane
// (Eq. InstFlux) and the wall-normal viscous stress n^T S n.
#include "internal.cuh"

namespace mafp {

constexpr int kPostThreads = 256;

// Film particles: v <- v + dt (-eta / (rho H^2) v - grad p / rho + g_par), then
// v is projected onto the tangent plane (film velocity is parallel to the
// surface).  grad p is the applied gradient of field 3 (the pressure slot).
// Particles with H <= 0 keep their velocity.
template <typename T>
__global__ void k_film_momentum(int64_t n, const uint8_t *model, vec4_t<T> *vp, const T *rho,
                                const T *eta, const T *hfilm, const vec4_t<T> *normal,
                                const vec4_t<T> *out, double gx, double gy, double gz,
                                double dt) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    if (model[i] != MAFP_MODEL_2D) continue;
    const double H = (double)hfilm[i];
    if (!(H > 0.0)) continue;
    vec4_t<T> v = ld4(vp + i);
    const vec4_t<T> nn = ld4(normal + i);
    const vec4_t<T> gp = ld4(out + 4 * i + 3);     // (d/dx, d/dy, d/dz, Lap) of p
    const double r = (double)rho[i];
    const double damp = (double)eta[i] / (r * H * H);
    const double gn = gx * nn.x + gy * nn.y + gz * nn.z;
    const double gpx = gx - gn * nn.x, gpy = gy - gn * nn.y, gpz = gz - gn * nn.z;
    double vx = v.x + dt * (-damp * v.x - gp.x / r + gpx);
    double vy = v.y + dt * (-damp * v.y - gp.y / r + gpy);
    double vz = v.z + dt * (-damp * v.z - gp.z / r + gpz);
    const double vn = vx * nn.x + vy * nn.y + vz * nn.z;
    vx -= vn * nn.x;
    vy -= vn * nn.y;
    vz -= vn * nn.z;
    v.x = (T)vx;
    v.y = (T)vy;
    v.z = (T)vz;
    st4(vp + i, v);
  }
}

// Flux through the plane (point c, unit normal m) over one step: every
// particle whose signed distance goes from < 0 to >= 0 adds its volume m/rho,
// every one going back subtracts it.  out[0] += the sum, out[1] += crossings.
template <typename T>
__global__ void k_plane_flux(int64_t n, const vec4_t<T> *p0, const vec4_t<T> *p1, const T *mass,
                             const T *rho, double cx, double cy, double cz, double mx, double my,
                             double mz, double *out) {
  double s = 0.0, cnt = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const vec4_t<T> a = ld4(p0 + i), b = ld4(p1 + i);
    const double da = (a.x - cx) * mx + (a.y - cy) * my + (a.z - cz) * mz;
    const double db = (b.x - cx) * mx + (b.y - cy) * my + (b.z - cz) * mz;
    const double vol = (double)mass[i] / (double)rho[i];
    if (da < 0.0 && db >= 0.0) {
      s += vol;
      cnt += 1.0;
    } else if (da >= 0.0 && db < 0.0) {
      s -= vol;
      cnt += 1.0;
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    s += __shfl_xor_sync(0xffffffffu, s, o);
    cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
  }
  if ((threadIdx.x & 31) == 0 && (s != 0.0 || cnt != 0.0)) {
    atomicAdd(out, s);
    atomicAdd(out + 1, cnt);
  }
}

// n^T S n = 2 eta n^T (grad v) n for S = eta (grad v + grad v^T), from the
// applied gradients of the velocity fields 0..2: (grad v)_{ab} = d v_a / d x_b
// = out[4i + a][b].  Summed over the selected particles: out[0] += sum,
// out[1] += count.
template <typename T>
__global__ void k_normal_stress(int64_t n, const uint8_t *select, const vec4_t<T> *out4,
                                const T *eta, const vec4_t<T> *normal, double *res) {
  double s = 0.0, cnt = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    if (!select[i]) continue;
    const vec4_t<T> nn = ld4(normal + i);
    const double nv[3] = {(double)nn.x, (double)nn.y, (double)nn.z};
    double q = 0.0;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const vec4_t<T> g = ld4(out4 + 4 * i + a);   // d v_a / d(x, y, z)
      q += nv[a] * (g.x * nv[0] + g.y * nv[1] + g.z * nv[2]);
    }
    s += 2.0 * (double)eta[i] * q;
    cnt += 1.0;
  }
  for (int o = 16; o > 0; o >>= 1) {
    s += __shfl_xor_sync(0xffffffffu, s, o);
    cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
  }
  if ((threadIdx.x & 31) == 0 && cnt != 0.0) {
    atomicAdd(res, s);
    atomicAdd(res + 1, cnt);
  }
}

int film_momentum(mafp_ctx *ctx, int64_t n, int32_t dtype, const uint8_t *model, void *vp,
                  const void *rho, const void *eta, const void *hfilm, const void *normal,
                  const void *out, const double *g, double dt, cudaStream_t s) {
  const int blocks = grid_for(n, kPostThreads, sm_count() * 16);
  if (dtype == MAFP_F64) {
    MAFP_TIMED(ctx, s, "k_film_momentum<double>",
               k_film_momentum<double><<<blocks, kPostThreads, 0, s>>>(
                   n, model, (double4_16a *)vp, (const double *)rho, (const double *)eta,
                   (const double *)hfilm, (const double4_16a *)normal, (const double4_16a *)out,
                   g[0], g[1], g[2], dt));
  } else {
    MAFP_TIMED(ctx, s, "k_film_momentum<float>",
               k_film_momentum<float><<<blocks, kPostThreads, 0, s>>>(
                   n, model, (float4 *)vp, (const float *)rho, (const float *)eta,
                   (const float *)hfilm, (const float4 *)normal, (const float4 *)out, g[0], g[1],
                   g[2], dt));
  }
  MAFP_LAUNCH_CHECK(ctx);
  return MAFP_OK;
}

int plane_flux(mafp_ctx *ctx, int64_t n, int32_t dtype, const void *p0, const void *p1,
               const void *mass, const void *rho, const double *c, const double *m, double *out,
               cudaStream_t s) {
  const int blocks = grid_for(n, kPostThreads, sm_count() * 8);
  if (dtype == MAFP_F64) {
    MAFP_TIMED(ctx, s, "k_plane_flux<double>",
               k_plane_flux<double><<<blocks, kPostThreads, 0, s>>>(
                   n, (const double4_16a *)p0, (const double4_16a *)p1, (const double *)mass,
                   (const double *)rho, c[0], c[1], c[2], m[0], m[1], m[2], out));
  } else {
    MAFP_TIMED(ctx, s, "k_plane_flux<float>",
               k_plane_flux<float><<<blocks, kPostThreads, 0, s>>>(
                   n, (const float4 *)p0, (const float4 *)p1, (const float *)mass,
                   (const float *)rho, c[0], c[1], c[2], m[0], m[1], m[2], out));
  }
  MAFP_LAUNCH_CHECK(ctx);
  return MAFP_OK;
}

int normal_stress(mafp_ctx *ctx, int64_t n, int32_t dtype, const uint8_t *select,
                  const void *out, const void *eta, const void *normal, double *res,
                  cudaStream_t s) {
  const int blocks = grid_for(n, kPostThreads, sm_count() * 8);
  if (dtype == MAFP_F64) {
    MAFP_TIMED(ctx, s, "k_normal_stress<double>",
               k_normal_stress<double><<<blocks, kPostThreads, 0, s>>>(
                   n, select, (const double4_16a *)out, (const double *)eta,
                   (const double4_16a *)normal, res));
  } else {
    MAFP_TIMED(ctx, s, "k_normal_stress<float>",
               k_normal_stress<float><<<blocks, kPostThreads, 0, s>>>(
                   n, select, (const float4 *)out, (const float *)eta, (const float4 *)normal,
                   res));
  }
  MAFP_LAUNCH_CHECK(ctx);
  return MAFP_OK;
}

}  // namespace mafp
