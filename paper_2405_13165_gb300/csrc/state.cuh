// state.cuh -- typed view of a mafp_state (the particle arrays a model
// transition reads and writes).
#pragma once
#include "internal.cuh"

namespace mafp {

template <typename T>
struct StateT {
  vec4_t<T> *pos_h, *vp, *normal;
  T *rho, *eta, *mass, *diam, *hfilm, *h3d;
  uint8_t *model, *type, *last;
};

template <typename T>
inline StateT<T> cast_state(const mafp_state *s) {
  StateT<T> r;
  r.pos_h = (vec4_t<T> *)s->pos_h;
  r.vp = (vec4_t<T> *)s->vp;
  r.normal = (vec4_t<T> *)s->normal;
  r.rho = (T *)s->rho;
  r.eta = (T *)s->eta;
  r.mass = (T *)s->mass;
  r.diam = (T *)s->diam;
  r.hfilm = (T *)s->hfilm;
  r.h3d = (T *)s->h3d;
  r.model = s->model;
  r.type = s->type;
  r.last = s->last;
  return r;
}

// Copy particle i of `a` to row o of `b`.
template <typename T>
__device__ __forceinline__ void copy_particle(const StateT<T> &a, int64_t i, const StateT<T> &b,
                                              int64_t o) {
  st4(b.pos_h + o, ld4(a.pos_h + i));
  st4(b.vp + o, ld4(a.vp + i));
  st4(b.normal + o, ld4(a.normal + i));
  b.rho[o] = a.rho[i];
  b.eta[o] = a.eta[i];
  b.mass[o] = a.mass[i];
  b.diam[o] = a.diam[i];
  b.hfilm[o] = a.hfilm[i];
  b.h3d[o] = a.h3d[i];
  b.model[o] = a.model[i];
  b.type[o] = a.type[i];
  b.last[o] = a.last[i];
}

}  // namespace mafp
