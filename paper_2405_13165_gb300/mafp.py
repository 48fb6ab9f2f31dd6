"""Thin ctypes binding of libmafp.so (include/mafp.h).

Argument marshalling only: every function checks tensor devices, dtypes and
contiguity, passes raw device pointers and the current CUDA stream, and raises
MafpError on a non-zero status.  All computation happens in the library's
CUDA kernels; there is no CPU fallback.  Names follow the C entry points.
"""
from __future__ import annotations

import ctypes as C
import math
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libmafp.so")

OK, EINVAL, ECAPACITY, ECUDA, ETIMEOUT, ENOTIMPL, ENONFINITE = 0, -1, -2, -3, -4, -5, -6
MAX_CLOUDS = 65536          # largest batch of mafp_build_neighbours_batched
F32_REFINED, F32_PLAIN, F64 = 0, 1, 2
MODEL_3D, MODEL_2D = 0, 1
TYPE_INTERIOR, TYPE_FREE_SURFACE, TYPE_WALL = 0, 1, 2
USER_TO_2D, USER_TO_3D = 1, 2
STENCIL_OK, STENCIL_DEFICIENT, STENCIL_FP64 = 0, 1, 2
_CODES = {0: "OK", -1: "EINVAL", -2: "ECAPACITY", -3: "ECUDA", -4: "ETIMEOUT", -5: "ENOTIMPL",
          -6: "ENONFINITE"}


class MafpError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"mafp error {_CODES.get(code, code)}: {msg}")
        self.code = code


class Params(C.Structure):
    _fields_ = [(k, C.c_double) for k in
                ("eps_lambda_max", "theta_star", "alpha_film", "alpha_w", "c_psi", "cond_fp64",
                 "eps_band", "angle_band", "hfilm_band", "near_rel", "wait_limit")]


class Status(C.Structure):
    _fields_ = [("code", C.c_int32), ("cells_identity", C.c_int32), ("required", C.c_int64),
                ("nnz", C.c_int64), ("n_fp64_stencil", C.c_int64), ("n_fp64_eigen", C.c_int64),
                ("n_deficient", C.c_int64), ("n_near", C.c_int64), ("n_out", C.c_int64),
                ("n_nonfinite", C.c_int64), ("ncells", C.c_int64), ("cell_size", C.c_double)]


class Tuning(C.Structure):
    _fields_ = [("stencil3d_group", C.c_int32), ("stencil2d_group", C.c_int32),
                ("apply_group", C.c_int32), ("grad3d_group", C.c_int32),
                ("grad2d_group", C.c_int32), ("cell_edge_pct", C.c_int32),
                ("classify_group", C.c_int32)]


class KernelTime(C.Structure):
    _fields_ = [("name", C.c_char * 64), ("launches", C.c_int64), ("total_ms", C.c_double)]


class State(C.Structure):
    _fields_ = [(k, C.c_void_p) for k in
                ("pos_h", "vp", "normal", "rho", "eta", "mass", "diam", "hfilm", "h3d",
                 "model", "type", "last")]


STATE_F4 = ("pos_h", "vp", "normal")
STATE_F1 = ("rho", "eta", "mass", "diam", "hfilm", "h3d")
STATE_U8 = ("model", "type", "last")

_lib = None


def lib():
    """Load libmafp.so; fail loudly when it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                               "`python -c 'import __graft_entry__ as g; g.build()'`")
        L = C.CDLL(LIB_PATH)
        p, i32, i64 = C.c_void_p, C.c_int32, C.c_int64
        L.mafp_default_params.argtypes = [p]
        L.mafp_create.argtypes = [p, p, i64, i64]
        L.mafp_destroy.argtypes = [p]
        L.mafp_last_error.argtypes = [p]
        L.mafp_last_error.restype = C.c_char_p
        L.mafp_get_status.argtypes = [p, p, p]
        L.mafp_reset_status.argtypes = [p, p]
        L.mafp_build_neighbours.argtypes = [p, i64, i32, p, p, p, i64, p, p, p]
        L.mafp_build_neighbours_batched.argtypes = [p, i64, i32, i32, p, p, p, p, i64, p, p, p]
        L.mafp_cell_order.argtypes = [p, i64, i32, p, p, p]
        L.mafp_ghost_sources.argtypes = [p, i64, p, p, p, p, p]
        L.mafp_ghost_seed.argtypes = [p, i64, i32, p, p, p, i64, p, p, p, p]
        L.mafp_ghost_append.argtypes = [p, i64, i64, i32, p, p, i64, p, p]
        L.mafp_film_momentum.argtypes = [p, i64, i32, p, p, p, p, p, p, p, p, C.c_double, p]
        L.mafp_plane_flux.argtypes = [p, i64, i32, p, p, p, p, p, p, p, p]
        L.mafp_normal_stress.argtypes = [p, i64, i32, p, p, p, p, p, p]
        L.mafp_classify_pca.argtypes = [p, i64, i32] + [p] * 17
        L.mafp_build_stencils.argtypes = [p, i64, i32, p, p, p, p, p, p, p, p, p]
        L.mafp_apply_ops.argtypes = [p, i64, i32, p, p, p, p, p, p]
        L.mafp_transpose_map.argtypes = [p, i64, p, p, p, p]
        L.mafp_apply_ops_backward.argtypes = [p, i64, i32, p, p, p, p, p, p, p]
        L.mafp_build_stencils_backward.argtypes = [p, i64, i32, p, p, p, p, p, p, p, p, p]
        L.mafp_remap_switched.argtypes = [p, i64, i32, p, p, p, p, p, i64, p, p, p]
        L.mafp_set_tuning.argtypes = [p, p]
        L.mafp_get_tuning.argtypes = [p, p]
        L.mafp_profile.argtypes = [p, i32]
        L.mafp_profile_read.argtypes = [p, p, i32, p]
        for name in ("mafp_set_tuning", "mafp_get_tuning", "mafp_profile", "mafp_profile_read", "mafp_create", "mafp_destroy", "mafp_get_status", "mafp_reset_status",
                     "mafp_build_neighbours", "mafp_build_neighbours_batched", "mafp_cell_order",
                     "mafp_classify_pca", "mafp_build_stencils",
                     "mafp_apply_ops", "mafp_transpose_map", "mafp_apply_ops_backward",
                     "mafp_build_stencils_backward", "mafp_remap_switched",
                     "mafp_ghost_sources", "mafp_ghost_seed", "mafp_ghost_append",
                     "mafp_film_momentum", "mafp_plane_flux", "mafp_normal_stress"):
            getattr(L, name).restype = C.c_int
        _lib = L
    return _lib


def default_params(**over) -> Params:
    p = Params()
    lib().mafp_default_params(C.byref(p))
    for k, v in over.items():
        setattr(p, k, float(v))
    return p


def real_dtype(dtype: int) -> torch.dtype:
    return torch.float64 if dtype == F64 else torch.float32


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _stream(stream):
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _need(t, name, dtype=None, numel=None, allow_none=False):
    if t is None:
        if allow_none:
            return
        raise ValueError(f"{name} is required")
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if dtype is not None and t.dtype != dtype:
        raise ValueError(f"{name} must be {dtype}, got {t.dtype}")
    if numel is not None and t.numel() < numel:
        raise ValueError(f"{name} needs at least {numel} elements, has {t.numel()}")


class Context:
    """Owns a mafp_ctx (device scratch sized for cap_particles / cap_cells)."""

    def __init__(self, cap_particles: int, cap_cells: int | None = None,
                 params: Params | None = None, device=None):
        if device is not None:
            torch.cuda.set_device(device)
        self.cap_particles = int(cap_particles)
        self.cap_cells = int(cap_cells if cap_cells is not None else
                             min(max(8 * cap_particles, 1 << 20), (1 << 31) - 2))
        self.params = params if params is not None else default_params()
        h = C.c_void_p()
        rc = lib().mafp_create(C.byref(h), C.byref(self.params), self.cap_particles, self.cap_cells)
        if rc != 0:
            raise MafpError(rc, "mafp_create failed")
        self.handle = h

    def close(self):
        if getattr(self, "handle", None):
            lib().mafp_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def check(self, rc):
        if rc != 0:
            raise MafpError(rc, lib().mafp_last_error(self.handle).decode())

    def status(self, stream=None) -> dict:
        st = Status()
        self.check(lib().mafp_get_status(self.handle, C.byref(st), _stream(stream)))
        return {k: getattr(st, k) for k, _ in Status._fields_}

    def tuning(self) -> dict:
        t = Tuning()
        self.check(lib().mafp_get_tuning(self.handle, C.byref(t)))
        return {k: getattr(t, k) for k, _ in Tuning._fields_}

    def set_tuning(self, **kw):
        cur = self.tuning()
        cur.update(kw)
        t = Tuning(**cur)
        self.check(lib().mafp_set_tuning(self.handle, C.byref(t)))

    def profile(self, enable: bool):
        """Start (clearing the record) or stop kernel-level event timing."""
        self.check(lib().mafp_profile(self.handle, 1 if enable else 0))

    def profile_read(self) -> dict:
        """{kernel name: (launches, total ms)} of the recorded launches."""
        buf = (KernelTime * 256)()
        cnt = C.c_int32(0)
        self.check(lib().mafp_profile_read(self.handle, buf, 256, C.byref(cnt)))
        return {buf[k].name.decode(): (int(buf[k].launches), float(buf[k].total_ms))
                for k in range(cnt.value)}

    def reset_status(self, stream=None):
        self.check(lib().mafp_reset_status(self.handle, _stream(stream)))


def build_neighbours(ctx: Context, pos_h, row_ptr, col, nnz=None, order=None, dtype=F32_REFINED,
                     stream=None):
    """Eq. Nbd neighbourhoods as CSR into caller buffers (see mafp.h)."""
    n = pos_h.shape[0]
    _need(pos_h, "pos_h", real_dtype(dtype), 4 * n)
    _need(row_ptr, "row_ptr", torch.int64, n + 1)
    _need(col, "col", torch.int32)
    _need(nnz, "nnz", torch.int64, 1, allow_none=True)
    _need(order, "order", torch.int32, n, allow_none=True)
    ctx.check(lib().mafp_build_neighbours(ctx.handle, n, dtype, _ptr(pos_h), _ptr(row_ptr),
                                          _ptr(col), col.numel(), _ptr(nnz), _ptr(order),
                                          _stream(stream)))


def cell_order(ctx: Context, pos_h, order, dtype=F32_REFINED, stream=None):
    """Permutation into cell order (order[s] = particle at sorted position s)."""
    n = pos_h.shape[0]
    _need(pos_h, "pos_h", real_dtype(dtype), 4 * n)
    _need(order, "order", torch.int32, n)
    ctx.check(lib().mafp_cell_order(ctx.handle, n, dtype, _ptr(pos_h), _ptr(order),
                                    _stream(stream)))


def build_neighbours_batched(ctx: Context, cloud_offset, pos_h, row_ptr, col, nnz=None, order=None,
                             dtype=F32_REFINED, stream=None):
    """Eq. Nbd for clouds stored back to back, cloud b = [offset[b], offset[b+1])."""
    n = pos_h.shape[0]
    nb = cloud_offset.numel() - 1
    _need(cloud_offset, "cloud_offset", torch.int64, nb + 1)
    _need(pos_h, "pos_h", real_dtype(dtype), 4 * n)
    _need(row_ptr, "row_ptr", torch.int64, n + 1)
    _need(col, "col", torch.int32)
    _need(nnz, "nnz", torch.int64, 1, allow_none=True)
    _need(order, "order", torch.int32, n, allow_none=True)
    ctx.check(lib().mafp_build_neighbours_batched(ctx.handle, n, dtype, nb, _ptr(cloud_offset),
                                                  _ptr(pos_h), _ptr(row_ptr), _ptr(col),
                                                  col.numel(), _ptr(nnz), _ptr(order),
                                                  _stream(stream)))


def neighbours(ctx: Context, pos_h, dtype=F32_REFINED, cap_nnz=None, order=False, stream=None):
    """Allocating convenience form: returns (row_ptr, col[:nnz], order or None)."""
    n = pos_h.shape[0]
    dev = pos_h.device
    row_ptr = torch.empty(n + 1, dtype=torch.int64, device=dev)
    nnz = torch.zeros(1, dtype=torch.int64, device=dev)
    cap = int(cap_nnz) if cap_nnz is not None else max(256 * n, 1)
    col = torch.empty(cap, dtype=torch.int32, device=dev)
    od = torch.empty(n, dtype=torch.int32, device=dev) if order else None
    ctx.reset_status(stream)
    build_neighbours(ctx, pos_h, row_ptr, col, nnz, od, dtype, stream)
    st = ctx.status(stream)
    if st["code"] != 0:
        raise MafpError(st["code"], f"device status after build_neighbours: {st}")
    return row_ptr, col[: int(nnz.item())], od


def classify_pca(ctx: Context, pos_h, model, ptype, normal, vol, h3d, user, last, row_ptr, col,
                 flag, preflag, eig, frame, hfilm, near=None, dtype=F32_REFINED, stream=None):
    n = pos_h.shape[0]
    rd = real_dtype(dtype)
    _need(pos_h, "pos_h", rd, 4 * n)
    for t, nm in ((model, "model"), (ptype, "type"), (user, "user"), (last, "last"),
                  (flag, "flag"), (preflag, "preflag")):
        _need(t, nm, torch.uint8, n)
    _need(near, "near", torch.uint8, n, allow_none=True)
    _need(normal, "normal", rd, 4 * n)
    _need(vol, "vol", rd, n)
    _need(h3d, "h3d", rd, n)
    _need(eig, "eig", rd, 4 * n)
    _need(frame, "frame", rd, 8 * n)
    _need(hfilm, "hfilm", rd, n)
    _need(row_ptr, "row_ptr", torch.int64, n + 1)
    _need(col, "col", torch.int32)
    ctx.check(lib().mafp_classify_pca(ctx.handle, n, dtype, _ptr(pos_h), _ptr(model), _ptr(ptype),
                                      _ptr(normal), _ptr(vol), _ptr(h3d), _ptr(user), _ptr(last),
                                      _ptr(row_ptr), _ptr(col), _ptr(flag), _ptr(preflag),
                                      _ptr(eig), _ptr(frame), _ptr(hfilm), _ptr(near),
                                      _stream(stream)))


def build_stencils(ctx: Context, pos_h, model, frame, row_ptr, col, coef, status, cond,
                   dtype=F32_REFINED, stream=None):
    n = pos_h.shape[0]
    rd = real_dtype(dtype)
    _need(pos_h, "pos_h", rd, 4 * n)
    _need(model, "model", torch.uint8, n)
    _need(frame, "frame", rd, 8 * n)
    _need(row_ptr, "row_ptr", torch.int64, n + 1)
    _need(col, "col", torch.int32)
    _need(coef, "coef", rd, 4 * col.numel())
    _need(status, "status", torch.uint8, n)
    _need(cond, "cond", torch.float32, n)
    ctx.check(lib().mafp_build_stencils(ctx.handle, n, dtype, _ptr(pos_h), _ptr(model), _ptr(frame),
                                        _ptr(row_ptr), _ptr(col), _ptr(coef), _ptr(status),
                                        _ptr(cond), _stream(stream)))


def apply_ops(ctx: Context, row_ptr, col, coef, fields, out, dtype=F32_REFINED, stream=None):
    n = row_ptr.numel() - 1
    rd = real_dtype(dtype)
    _need(row_ptr, "row_ptr", torch.int64)
    _need(col, "col", torch.int32)
    _need(coef, "coef", rd, 4 * col.numel())
    _need(fields, "fields", rd, 4 * n)
    _need(out, "out", rd, 16 * n)
    ctx.check(lib().mafp_apply_ops(ctx.handle, n, dtype, _ptr(row_ptr), _ptr(col), _ptr(coef),
                                   _ptr(fields), _ptr(out), _stream(stream)))


def transpose_map(ctx: Context, row_ptr, col, tloc, stream=None):
    n = row_ptr.numel() - 1
    _need(row_ptr, "row_ptr", torch.int64)
    _need(col, "col", torch.int32)
    _need(tloc, "tloc", None, col.numel())
    if tloc.element_size() != 2:
        raise ValueError("tloc must hold 16-bit entries (torch.int16 or torch.uint16)")
    ctx.check(lib().mafp_transpose_map(ctx.handle, n, _ptr(row_ptr), _ptr(col), _ptr(tloc),
                                       _stream(stream)))


def apply_ops_backward(ctx: Context, row_ptr, col, tloc, coef, gout, gfields, dtype=F32_REFINED,
                       stream=None):
    """Adjoint of apply_ops w.r.t. the fields; tloc None scatters with atomics."""
    n = row_ptr.numel() - 1
    rd = real_dtype(dtype)
    _need(row_ptr, "row_ptr", torch.int64)
    _need(col, "col", torch.int32)
    _need(tloc, "tloc", None, col.numel(), allow_none=True)
    _need(coef, "coef", rd, 4 * col.numel())
    _need(gout, "gout", rd, 16 * n)
    _need(gfields, "gfields", rd, 4 * n)
    ctx.check(lib().mafp_apply_ops_backward(ctx.handle, n, dtype, _ptr(row_ptr), _ptr(col),
                                            _ptr(tloc), _ptr(coef), _ptr(gout), _ptr(gfields),
                                            _stream(stream)))


def build_stencils_backward(ctx: Context, pos_h, model, frame, row_ptr, col, fields, gout, gpos,
                            dtype=F32_REFINED, stream=None):
    n = pos_h.shape[0]
    rd = real_dtype(dtype)
    _need(pos_h, "pos_h", rd, 4 * n)
    _need(model, "model", torch.uint8, n)
    _need(frame, "frame", rd, 8 * n)
    _need(row_ptr, "row_ptr", torch.int64, n + 1)
    _need(col, "col", torch.int32)
    _need(fields, "fields", rd, 4 * n)
    _need(gout, "gout", rd, 16 * n)
    _need(gpos, "gpos", rd, 4 * n)
    ctx.check(lib().mafp_build_stencils_backward(ctx.handle, n, dtype, _ptr(pos_h), _ptr(model),
                                                 _ptr(frame), _ptr(row_ptr), _ptr(col),
                                                 _ptr(fields), _ptr(gout), _ptr(gpos),
                                                 _stream(stream)))


def make_state(arrays: dict, dtype=F32_REFINED) -> tuple[State, dict]:
    """Pack a dict of device tensors (pos_h, vp, normal, rho, eta, mass, diam,
    hfilm, h3d, model, type, last) into a mafp_state; returns (state, keep-alive)."""
    rd = real_dtype(dtype)
    for k in STATE_F4 + STATE_F1:
        _need(arrays[k], k, rd)
    for k in STATE_U8:
        _need(arrays[k], k, torch.uint8)
    st = State(**{k: arrays[k].data_ptr() for k in STATE_F4 + STATE_F1 + STATE_U8})
    return st, arrays


def remap_switched(ctx: Context, n: int, state_in: dict, flag, row_ptr, col, state_out: dict,
                   cap_out: int, old2new, n_out, dtype=F32_REFINED, stream=None):
    sin, _a = make_state(state_in, dtype)
    sout, _b = make_state(state_out, dtype)
    _need(flag, "flag", torch.uint8, n)
    _need(row_ptr, "row_ptr", torch.int64, n + 1)
    _need(col, "col", torch.int32)
    _need(old2new, "old2new", torch.int32, n)
    _need(n_out, "n_out", torch.int64, 1, allow_none=True)
    ctx.check(lib().mafp_remap_switched(ctx.handle, n, dtype, C.byref(sin), _ptr(flag),
                                        _ptr(row_ptr), _ptr(col), C.byref(sout), int(cap_out),
                                        _ptr(old2new), _ptr(n_out), _stream(stream)))


def symbols_declared_in_header(header: str | None = None) -> list[str]:
    """Names of the functions include/mafp.h declares (for the load test)."""
    import re
    header = header or os.path.join(os.path.dirname(_HERE), "include", "mafp.h")
    src = open(header).read()
    return sorted(set(re.findall(r"^\s*(?:int|void|const char \*)\s*(mafp_\w+)\s*\(", src, re.M)))


def ghost_sources(ctx: Context, model, row_ptr, col, src, stream=None):
    """Alg. 5, first loop: src[i] = 1 when S_i holds a particle of the other model."""
    n = row_ptr.numel() - 1
    _need(model, "model", torch.uint8, n)
    _need(row_ptr, "row_ptr", torch.int64, n + 1)
    _need(col, "col", torch.int32)
    _need(src, "src", torch.uint8, n)
    ctx.check(lib().mafp_ghost_sources(ctx.handle, n, _ptr(model), _ptr(row_ptr), _ptr(col),
                                       _ptr(src), _stream(stream)))


def ghost_seed(ctx: Context, n: int, state_in: dict, src, ghost: dict, cap_ghost: int,
               ghost_flag, ghost_src, n_ghost, dtype=F32_REFINED, stream=None):
    """Alg. 5, second loop: copies of the sources and the transition each takes."""
    sin, _a = make_state(state_in, dtype)
    sg, _b = make_state(ghost, dtype)
    _need(src, "src", torch.uint8, n)
    _need(ghost_flag, "ghost_flag", torch.uint8, cap_ghost)
    _need(ghost_src, "ghost_src", torch.int32, cap_ghost)
    _need(n_ghost, "n_ghost", torch.int64, 1, allow_none=True)
    ctx.check(lib().mafp_ghost_seed(ctx.handle, n, dtype, C.byref(sin), _ptr(src), C.byref(sg),
                                    int(cap_ghost), _ptr(ghost_flag), _ptr(ghost_src),
                                    _ptr(n_ghost), _stream(stream)))


def ghost_append(ctx: Context, n_regular: int, n_ghost: int, ghost: dict, all_: dict,
                 cap_all: int, n_all, dtype=F32_REFINED, stream=None):
    """Alg. 5 result: transitioned ghosts appended behind the regular particles."""
    sg, _a = make_state(ghost, dtype)
    sa, _b = make_state(all_, dtype)
    _need(n_all, "n_all", torch.int64, 1, allow_none=True)
    ctx.check(lib().mafp_ghost_append(ctx.handle, int(n_regular), int(n_ghost), dtype,
                                      C.byref(sg), C.byref(sa), int(cap_all), _ptr(n_all),
                                      _stream(stream)))


def _d3(v):
    a = (C.c_double * 3)(*[float(x) for x in v])
    return a


def film_momentum(ctx: Context, model, vp, rho, eta, hfilm, normal, out, gravity, dt: float,
                  dtype=F32_REFINED, stream=None):
    """Eq. FilmMomentum, explicit step for the film particles (vp updated in place)."""
    n = model.numel()
    rd = real_dtype(dtype)
    _need(model, "model", torch.uint8, n)
    for t, nm, k in ((vp, "vp", 4), (normal, "normal", 4), (out, "out", 16)):
        _need(t, nm, rd, k * n)
    for t, nm in ((rho, "rho"), (eta, "eta"), (hfilm, "hfilm")):
        _need(t, nm, rd, n)
    g = _d3(gravity)
    ctx.check(lib().mafp_film_momentum(ctx.handle, n, dtype, _ptr(model), _ptr(vp), _ptr(rho),
                                       _ptr(eta), _ptr(hfilm), _ptr(normal), _ptr(out), g,
                                       float(dt), _stream(stream)))


def plane_flux(ctx: Context, pos_old, pos_new, mass, rho, point, normal, acc,
               dtype=F32_REFINED, stream=None):
    """Volume through a plane over one step, accumulated into acc[0:2] (float64, device)."""
    n = pos_old.shape[0]
    rd = real_dtype(dtype)
    _need(pos_old, "pos_old", rd, 4 * n)
    _need(pos_new, "pos_new", rd, 4 * n)
    _need(mass, "mass", rd, n)
    _need(rho, "rho", rd, n)
    _need(acc, "acc", torch.float64, 2)
    ctx.check(lib().mafp_plane_flux(ctx.handle, n, dtype, _ptr(pos_old), _ptr(pos_new),
                                    _ptr(mass), _ptr(rho), _d3(point), _d3(normal), _ptr(acc),
                                    _stream(stream)))


def normal_stress(ctx: Context, select, out, eta, normal, acc, dtype=F32_REFINED, stream=None):
    """Sum and count of n^T S n over the selected particles into acc[0:2] (float64, device)."""
    n = select.numel()
    rd = real_dtype(dtype)
    _need(select, "select", torch.uint8, n)
    _need(out, "out", rd, 16 * n)
    _need(eta, "eta", rd, n)
    _need(normal, "normal", rd, 4 * n)
    _need(acc, "acc", torch.float64, 2)
    ctx.check(lib().mafp_normal_stress(ctx.handle, n, dtype, _ptr(select), _ptr(out), _ptr(eta),
                                       _ptr(normal), _ptr(acc), _stream(stream)))
