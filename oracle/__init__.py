"""Python front-end of the plain FP64 CPU oracle (``oracle.c``).

TEST INFRASTRUCTURE ONLY: the test-suite, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg are the only callers.  Nothing here touches the
CUDA library; inputs are promoted to float64 before the C code sees them.
"""
from __future__ import annotations

import ctypes as C
import math
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lib = None

DEFAULT_PARAMS = dict(
    eps_lambda_max=0.15,        # Sec. 4.1.2
    theta_star=math.pi / 6.0,   # Sec. 4.1.3
    alpha_film=4.0,             # Eq. Height (alpha not given in the paper)
    alpha_w=4.0,                # GFDM weight shape (not given)
    c_psi=1.0 / 3.5,            # (r_min + r_max)/2 of Sec. 5.2 (not given)
    near_rel=1e-6,              # near-threshold reporting band
)


class _Params(C.Structure):
    _fields_ = [(k, C.c_double) for k in DEFAULT_PARAMS]


class _State(C.Structure):
    _fields_ = [(k, C.c_void_p) for k in
                ("pos_h", "vp", "normal", "rho", "eta", "mass", "diam", "hfilm", "h3d",
                 "model", "type", "last")]


STATE_KEYS_F4 = ("pos_h", "vp", "normal")
STATE_KEYS_F1 = ("rho", "eta", "mass", "diam", "hfilm", "h3d")
STATE_KEYS_U8 = ("model", "type", "last")


def build(force: bool = False) -> str:
    """Compile liboracle.so next to the sources (plain C, OpenMP over particles)."""
    src = os.path.join(_HERE, "oracle.c")
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < max(
            os.path.getmtime(src), os.path.getmtime(os.path.join(_HERE, "oracle.h"))):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fno-fast-math", "-ffp-contract=off", "-fopenmp",
                               "-fPIC", "-shared", "-std=c11", "-D_DEFAULT_SOURCE", src,
                               "-o", tmp, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB_PATH)
        p, i64, i32 = C.c_void_p, C.c_int64, C.c_int32
        L.orc_in_support.argtypes = [p, i64, i64]
        L.orc_row_brute.argtypes = [i64, p, i64, p]
        L.orc_row_brute.restype = i64
        L.orc_neighbours.argtypes = [i64, p, p, p, i64]
        L.orc_neighbours.restype = i64
        L.orc_jacobi3.argtypes = [p, p, p]
        L.orc_pca.argtypes = [p, p, p, p, i64, p, p]
        L.orc_pca.restype = i64
        L.orc_classify.argtypes = [i64, p, p, p, p, p, p, p, p, p, p, p, i64, p, p, p, p, p]
        L.orc_smooth.argtypes = [i64, p, p, p, p, p, p, i64, p]
        L.orc_stencils.argtypes = [i64, p, p, p, p, p, p, i64, p, p, p]
        L.orc_apply.argtypes = [i64, p, p, p, p, p, i64, p]
        L.orc_apply_T.argtypes = [i64, p, p, p, p, p]
        L.orc_remap.argtypes = [i64, p, p, p, p, p, p, i64, p]
        L.orc_stencil_grad.argtypes = [i64, p, p, p, p, p, p, p, p]
        L.orc_remap.restype = i64
        L.orc_ghost_sources.argtypes = [i64, p, p, p, p]
        _lib = L
    return _lib


def set_threads(n: int) -> None:
    """Limit the OpenMP threads of later oracle calls."""
    try:
        omp = C.CDLL("libgomp.so.1")
        omp.omp_set_num_threads(int(n))
    except OSError:
        pass


def _f64(a, cols=None):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    if cols is not None:
        a = a.reshape(-1, cols)
    return a


def _u8(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.uint8))


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _params(prm):
    d = dict(DEFAULT_PARAMS)
    if prm:
        d.update(prm)
    return _Params(**d)


def _rows(rows):
    if rows is None:
        return None, 0
    r = np.ascontiguousarray(np.asarray(rows, dtype=np.int64))
    return r, r.size


def in_support(pos_h, i, j) -> bool:
    P = _f64(pos_h, 4)
    return bool(lib().orc_in_support(_ptr(P), int(i), int(j)))


def row_brute(pos_h, i) -> np.ndarray:
    """S_i by brute force over all particles (Eq. Nbd)."""
    P = _f64(pos_h, 4)
    n = P.shape[0]
    k = lib().orc_row_brute(n, _ptr(P), int(i), None)
    out = np.empty(k, np.int32)
    lib().orc_row_brute(n, _ptr(P), int(i), _ptr(out))
    return out


def neighbours(pos_h):
    """All rows S_i as CSR (row_ptr int64 [n+1], col int32 [nnz])."""
    P = _f64(pos_h, 4)
    n = P.shape[0]
    row_ptr = np.zeros(n + 1, np.int64)
    nnz = lib().orc_neighbours(n, _ptr(P), _ptr(row_ptr), None, 0)
    col = np.empty(max(int(row_ptr[-1]), 1), np.int32)
    nnz = lib().orc_neighbours(n, _ptr(P), _ptr(row_ptr), _ptr(col), col.size)
    assert nnz == row_ptr[-1]
    return row_ptr, col[:nnz]


def jacobi3(A):
    A = _f64(A).reshape(9).copy()
    lam = np.zeros(3)
    V = np.zeros(9)
    lib().orc_jacobi3(_ptr(A), _ptr(lam), _ptr(V))
    return lam, V.reshape(3, 3)


def pca(pos_h, model, row_ptr, col, i):
    P = _f64(pos_h, 4)
    lam = np.zeros(3)
    V = np.zeros(9)
    m = lib().orc_pca(_ptr(P), _ptr(_u8(model)), _ptr(np.ascontiguousarray(row_ptr, np.int64)),
                      _ptr(np.ascontiguousarray(col, np.int32)), int(i), _ptr(lam), _ptr(V))
    return m, lam, V.reshape(3, 3)


def classify(pos_h, model, ptype, normal, vol, h3d, user, row_ptr, col, rows=None, prm=None):
    """Pre-flags of Sec. 4 (before smoothing) plus PCA and film-height outputs."""
    P = _f64(pos_h, 4)
    n = P.shape[0]
    N = _f64(normal, 4)
    r, nr = _rows(rows)
    pre = np.zeros(n, np.uint8)
    near = np.zeros(n, np.uint8)
    eig = np.zeros((n, 4))
    frame = np.zeros((n, 8))
    hf = np.zeros(n)
    pr = _params(prm)
    lib().orc_classify(n, _ptr(P), _ptr(_u8(model)), _ptr(_u8(ptype)), _ptr(N), _ptr(_f64(vol)),
                       _ptr(_f64(h3d)), _ptr(_u8(user)),
                       _ptr(np.ascontiguousarray(row_ptr, np.int64)),
                       _ptr(np.ascontiguousarray(col, np.int32)), C.byref(pr), _ptr(r), nr,
                       _ptr(pre), _ptr(eig), _ptr(frame), _ptr(hf), _ptr(near))
    return dict(preflag=pre, eig=eig, frame=frame, hfilm=hf, near=near)


def smooth(model, preflag, last, row_ptr, col, rows=None):
    n = len(model)
    r, nr = _rows(rows)
    flag = np.zeros(n, np.uint8)
    lib().orc_smooth(n, _ptr(_u8(model)), _ptr(_u8(preflag)), _ptr(_u8(last)),
                     _ptr(np.ascontiguousarray(row_ptr, np.int64)),
                     _ptr(np.ascontiguousarray(col, np.int32)), _ptr(r), nr, _ptr(flag))
    return flag


def stencils(pos_h, model, row_ptr, col, rows=None, prm=None):
    """GFDM coefficients [nnz,4] (c^x, c^y, c^z, c^Lap), status [n], cond [n]."""
    P = _f64(pos_h, 4)
    n = P.shape[0]
    row_ptr = np.ascontiguousarray(row_ptr, np.int64)
    r, nr = _rows(rows)
    coef = np.zeros((max(int(row_ptr[-1]), 1), 4))
    status = np.zeros(n, np.uint8)
    cond = np.zeros(n)
    pr = _params(prm)
    lib().orc_stencils(n, _ptr(P), _ptr(_u8(model)), _ptr(row_ptr),
                       _ptr(np.ascontiguousarray(col, np.int32)), C.byref(pr), _ptr(r), nr,
                       _ptr(coef), _ptr(status), _ptr(cond))
    return coef[: int(row_ptr[-1])], status, cond


def apply(row_ptr, col, coef, fields, rows=None):
    """out [n,4,4]: out[i, f] = (d_x, d_y, d_z, Lap) of field f at particle i."""
    row_ptr = np.ascontiguousarray(row_ptr, np.int64)
    n = row_ptr.size - 1
    F = _f64(fields, 4)
    cf = _f64(coef, 4) if len(coef) else np.zeros((1, 4))
    r, nr = _rows(rows)
    out = np.zeros((n, 4, 4))
    lib().orc_apply(n, _ptr(row_ptr), _ptr(np.ascontiguousarray(col, np.int32)), _ptr(cf),
                    _ptr(F), _ptr(r), nr, _ptr(out))
    return out


def apply_T(row_ptr, col, coef, gout):
    row_ptr = np.ascontiguousarray(row_ptr, np.int64)
    n = row_ptr.size - 1
    G = _f64(gout).reshape(n, 4, 4)
    cf = _f64(coef, 4) if len(coef) else np.zeros((1, 4))
    gf = np.zeros((n, 4))
    lib().orc_apply_T(n, _ptr(row_ptr), _ptr(np.ascontiguousarray(col, np.int32)), _ptr(cf),
                      _ptr(np.ascontiguousarray(G)), _ptr(gf))
    return gf


def stencil_grad(pos_h, model, row_ptr, col, fields, gout, prm=None):
    """dL/dx [n,4] through the stencils, given gout = dL/dout [n,4,4]."""
    P = _f64(pos_h, 4)
    n = P.shape[0]
    F = _f64(fields, 4)
    G = np.ascontiguousarray(_f64(gout).reshape(n, 4, 4))
    g = np.zeros((n, 4))
    pr = _params(prm)
    lib().orc_stencil_grad(n, _ptr(P), _ptr(_u8(model)),
                           _ptr(np.ascontiguousarray(row_ptr, np.int64)),
                           _ptr(np.ascontiguousarray(col, np.int32)), C.byref(pr), _ptr(F),
                           _ptr(G), _ptr(g))
    return g


def _state_arrays(st: dict, n: int):
    arrs = {}
    for k in STATE_KEYS_F4:
        arrs[k] = _f64(st[k], 4) if st is not None else np.zeros((n, 4))
    for k in STATE_KEYS_F1:
        arrs[k] = _f64(st[k]) if st is not None else np.zeros(n)
    for k in STATE_KEYS_U8:
        arrs[k] = _u8(st[k if k != "type" else "ptype"]) if st is not None else np.zeros(n, np.uint8)
    s = _State(**{k: _ptr(arrs[k]) for k in arrs})
    return s, arrs


def remap(state: dict, flag, row_ptr, col, cap_out=None, prm=None):
    """Sec. 5 model transition.  `state` has pos_h, vp, normal, rho, eta, mass,
    diam, hfilm, h3d, model, ptype, last.  Returns (out dict, old2new, n_out)."""
    n = len(state["model"])
    sin, keep_in = _state_arrays(state, n)
    if cap_out is None:
        cap_out = n + 64
        while True:
            pr = _params(prm)
            sout, arr_out = _state_arrays(None, cap_out)
            o2n = np.zeros(n, np.int32)
            n_out = lib().orc_remap(n, C.byref(sin), _ptr(_u8(flag)),
                                    _ptr(np.ascontiguousarray(row_ptr, np.int64)),
                                    _ptr(np.ascontiguousarray(col, np.int32)), C.byref(pr),
                                    C.byref(sout), cap_out, _ptr(o2n))
            if n_out >= 0:
                break
            cap_out = -n_out
    else:
        pr = _params(prm)
        sout, arr_out = _state_arrays(None, cap_out)
        o2n = np.zeros(n, np.int32)
        n_out = lib().orc_remap(n, C.byref(sin), _ptr(_u8(flag)),
                                _ptr(np.ascontiguousarray(row_ptr, np.int64)),
                                _ptr(np.ascontiguousarray(col, np.int32)), C.byref(pr),
                                C.byref(sout), cap_out, _ptr(o2n))
        if n_out < 0:
            return None, o2n, n_out
    out = {k: v[:n_out] for k, v in arr_out.items()}
    out["ptype"] = out.pop("type")
    return out, o2n, n_out


def cloud_state(cloud) -> dict:
    """State dict of a generated Cloud for `remap`."""
    return dict(pos_h=cloud.pos_h, vp=cloud.vp, normal=cloud.normal, rho=cloud.rho,
                eta=cloud.eta, mass=cloud.mass, diam=cloud.diam, hfilm=cloud.hfilm,
                h3d=cloud.h3d, model=cloud.model, ptype=cloud.ptype, last=cloud.last)


def pipeline(cloud, prm=None, rows=None):
    """Neighbours -> detection -> smoothing -> stencils -> application, FP64."""
    rp, col = neighbours(cloud.pos_h)
    cl = classify(cloud.pos_h, cloud.model, cloud.ptype, cloud.normal, cloud.vol, cloud.h3d,
                  cloud.user, rp, col, rows=None, prm=prm)
    flag = smooth(cloud.model, cl["preflag"], cloud.last, rp, col)
    coef, status, cond = stencils(cloud.pos_h, cloud.model, rp, col, rows=rows, prm=prm)
    out = apply(rp, col, coef, cloud.vp, rows=rows)
    return dict(row_ptr=rp, col=col, flag=flag, coef=coef, status=status, cond=cond, out=out, **cl)


def ghost_sources(model, row_ptr, col):
    """Alg. 5, first loop: 1 where S_i holds a particle of the other model."""
    n = len(model)
    src = np.zeros(n, np.uint8)
    lib().orc_ghost_sources(n, _ptr(_u8(model)), _ptr(np.ascontiguousarray(row_ptr, np.int64)),
                            _ptr(np.ascontiguousarray(col, np.int32)), _ptr(src))
    return src


def ghost_zone(state: dict, row_ptr, col, prm=None):
    """Alg. 5 on a cloud with its neighbour lists: sources, one ghost per source
    (same model, place and data), model transition of the ghosts (Alg. 3 for
    the 3D ghosts, walls flagged, interior / free-surface ghosts as candidates;
    Alg. 4 for the 2D ghosts), keeping the ghosts that transition produced.
    Returns (union state: regular particles then ghosts, ghost sources, the
    intermediate ghost flags, n_ghost_intermediate)."""
    model = np.asarray(state["model"])
    src = ghost_sources(model, row_ptr, col)
    idx = np.nonzero(src)[0]
    ghost = {k: np.array(v)[idx] for k, v in state.items()}
    ghost["last"] = np.zeros(idx.size, np.uint8)
    gm, gt = ghost["model"], ghost["ptype"]
    gflag = np.where(gm == 1, 2, np.where(gt == 2, 1, 0)).astype(np.uint8)
    grp, gcol = neighbours(ghost["pos_h"])
    out, _, n_out = remap(ghost, gflag, grp, gcol, prm=prm)
    keep = out["last"] == 1
    union = {k: np.concatenate([np.asarray(state[k]), np.asarray(out[k])[keep].astype(
        np.asarray(state[k]).dtype)]) for k in state}
    return union, src, gflag, idx.size


def film_momentum(model, vp, rho, eta, hfilm, normal, out, gravity, dt):
    """Eq. FilmMomentum, one explicit step for the 2D particles in FP64:
    v + dt (-eta / (rho H^2) v - grad p / rho + g_par), g_par = g - (g.n) n, then
    projected onto the tangent plane; grad p = out[i, 3, :3].  Particles with
    H <= 0 and 3D particles keep their velocity.  Returns the new vp."""
    vp = np.array(vp, np.float64)
    model = np.asarray(model)
    H = np.asarray(hfilm, np.float64)
    live = (model == 1) & (H > 0)
    n = np.asarray(normal, np.float64)[:, :3]
    r = np.asarray(rho, np.float64)
    e = np.asarray(eta, np.float64)
    gp = np.asarray(out, np.float64).reshape(-1, 4, 4)[:, 3, :3]
    g = np.asarray(gravity, np.float64)
    gpar = g[None, :] - (n @ g)[:, None] * n
    Hs = np.where(live, H, 1.0)
    v = vp[:, :3] + dt * (-(e / (r * Hs * Hs))[:, None] * vp[:, :3] - gp / r[:, None] + gpar)
    v = v - (v * n).sum(1)[:, None] * n
    vp[live, :3] = v[live]
    return vp


def plane_flux(pos_old, pos_new, mass, rho, point, normal):
    """Volume crossing a plane over one step (Eq. InstFlux as a sum over
    particles): + m/rho for a signed distance going from < 0 to >= 0, - m/rho
    back.  Returns (volume, crossings)."""
    c = np.asarray(point, np.float64)
    m = np.asarray(normal, np.float64)
    da = (np.asarray(pos_old, np.float64)[:, :3] - c) @ m
    db = (np.asarray(pos_new, np.float64)[:, :3] - c) @ m
    vol = np.asarray(mass, np.float64) / np.asarray(rho, np.float64)
    up = (da < 0) & (db >= 0)
    down = (da >= 0) & (db < 0)
    return float(vol[up].sum() - vol[down].sum()), int(up.sum() + down.sum())


def normal_stress(select, out, eta, normal):
    """Sum over the selected particles of n^T S n = 2 eta n^T (grad v) n with
    (grad v)_ab = out[i, a, b] (a = velocity component, b = derivative
    direction).  Returns (sum, count)."""
    sel = np.asarray(select).astype(bool)
    G = np.asarray(out, np.float64).reshape(-1, 4, 4)[sel, :3, :3]
    n = np.asarray(normal, np.float64)[sel, :3]
    q = np.einsum("ia,iab,ib->i", n, G, n)
    return float((2.0 * np.asarray(eta, np.float64)[sel] * q).sum()), int(sel.sum())
