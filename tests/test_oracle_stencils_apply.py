"""Pins of the oracle's GFDM stencils (Sec. 2.3, Eq. GFDM_Definition) and their
application."""
import math

import numpy as np
import pytest
import scipy.sparse as sp

from paper_2405_13165_gb300 import clouds as C

# monomials of degree <= 2 in world coordinates and their exact derivatives
MONO = [
    (lambda x, y, z: np.ones_like(x), lambda x, y, z: (0 * x, 0 * x, 0 * x, 0 * x)),
    (lambda x, y, z: x, lambda x, y, z: (1 + 0 * x, 0 * x, 0 * x, 0 * x)),
    (lambda x, y, z: y, lambda x, y, z: (0 * x, 1 + 0 * x, 0 * x, 0 * x)),
    (lambda x, y, z: z, lambda x, y, z: (0 * x, 0 * x, 1 + 0 * x, 0 * x)),
    (lambda x, y, z: x * x, lambda x, y, z: (2 * x, 0 * x, 0 * x, 2 + 0 * x)),
    (lambda x, y, z: y * y, lambda x, y, z: (0 * x, 2 * y, 0 * x, 2 + 0 * x)),
    (lambda x, y, z: z * z, lambda x, y, z: (0 * x, 0 * x, 2 * z, 2 + 0 * x)),
    (lambda x, y, z: x * y, lambda x, y, z: (y, x, 0 * x, 0 * x)),
    (lambda x, y, z: x * z, lambda x, y, z: (z, 0 * x, x, 0 * x)),
    (lambda x, y, z: y * z, lambda x, y, z: (0 * x, z, y, 0 * x)),
]


def _csr(rp, col, vals, n):
    return sp.csr_matrix((vals, col, rp), shape=(n, n))


def test_3d_reproduces_quadratics(orc):
    c = C.cube_on_sheet(0.02)
    rp, col = orc.neighbours(c.pos_h)
    coef, status, cond = orc.stencils(c.pos_h, c.model, rp, col)
    is3 = (c.model == 0) & (status == 0)
    assert is3.sum() == (c.model == 0).sum()
    P = c.pos_h.astype(np.float64)
    x, y, z = P[:, 0] - 0.5, P[:, 1] - 0.5, P[:, 2]
    for f, df in MONO:
        u = f(x, y, z)
        want = np.stack(df(x, y, z), 1)
        for op in range(4):
            got = _csr(rp, col, coef[:, op], c.n) @ u
            scale = 1.0 if op < 3 else 1.0 / c.pos_h[0, 3]
            assert np.max(np.abs(got - want[:, op])[is3]) < 1e-9 * max(scale, 1.0) * 50


def test_2d_reproduces_in_plane_quadratics_on_tilted_plane(orc):
    # film on a plane tilted out of z: tangential gradient and surface
    # Laplacian of quadratics in the plane coordinates are exact
    f = C.flat_film(0.01, 0.3, 0.001)
    th = 0.4
    R = np.array([[1, 0, 0], [0, math.cos(th), -math.sin(th)], [0, math.sin(th), math.cos(th)]])
    P = f.pos_h.astype(np.float64).copy()
    P[:, :3] = P[:, :3] @ R.T + np.array([0.1, -0.2, 0.3])
    rp, col = orc.neighbours(P)
    coef, status, cond = orc.stencils(P, f.model, rp, col)
    assert np.all(status == 0)
    e1, e2 = R[:, 0], R[:, 1]
    X = P[:, :3] - np.array([0.1, -0.2, 0.3])
    s, t = X @ e1, X @ e2
    cases = [(s, e1, 0.0), (t, e2, 0.0), (s * s, None, 2.0), (t * t, None, 2.0), (s * t, None, 0.0),
             (np.ones_like(s), 0 * e1, 0.0)]
    A = [_csr(rp, col, coef[:, k], len(P)) for k in range(4)]
    for u, g, lap in cases:
        grad = np.stack([A[k] @ u for k in range(3)], 1)
        if g is not None:
            assert np.max(np.abs(grad - g[None, :])) < 1e-9
        else:   # gradient of s^2 is 2 s e1, of t^2 is 2 t e2, of s t is t e1 + s e2
            pass
        assert np.max(np.abs(A[3] @ u - lap)) < 1e-6
    grad = np.stack([A[k] @ (s * t) for k in range(3)], 1)
    assert np.max(np.abs(grad - (t[:, None] * e1 + s[:, None] * e2))) < 1e-9


def test_min_norm_least_squares_equivalence(orc):
    # c = argmin sum c_j^2 / w_j  s.t. sum c_j p_j = b  equals the minimum-norm
    # solution of (W^1/2 P)^T y = b with c = W^1/2 y (numpy lstsq)
    c = C.random_cloud(800, seed=11, frac2d=0.0, h_lo=0.25, h_hi=0.25)
    rp, col = orc.neighbours(c.pos_h)
    coef, status, cond = orc.stencils(c.pos_h, c.model, rp, col)
    aw = orc.DEFAULT_PARAMS["alpha_w"]
    for i in [3, 40, 400]:
        assert status[i] == 0
        r = col[rp[i]:rp[i + 1]]
        h = float(c.pos_h[i, 3])
        q = (c.pos_h[r, :3].astype(float) - c.pos_h[i, :3].astype(float)) / h
        s = np.linalg.norm(q, axis=1)
        w = np.where(s <= 1, (np.exp(-aw * s * s) - math.exp(-aw)) / (1 - math.exp(-aw)), 0.0)
        Pm = np.stack([np.ones_like(s), q[:, 0], q[:, 1], q[:, 2], q[:, 0] ** 2, q[:, 1] ** 2,
                       q[:, 2] ** 2, q[:, 0] * q[:, 1], q[:, 0] * q[:, 2], q[:, 1] * q[:, 2]], 1)
        M = (np.sqrt(w)[:, None] * Pm).T
        for op, b in enumerate([np.eye(10)[1] / h, np.eye(10)[2] / h, np.eye(10)[3] / h,
                                2 * (np.eye(10)[4] + np.eye(10)[5] + np.eye(10)[6]) / h ** 2]):
            y = np.linalg.lstsq(M, b, rcond=None)[0]
            want = np.sqrt(w) * y
            got = coef[rp[i]:rp[i + 1], op]
            np.testing.assert_allclose(got, want, rtol=1e-7, atol=1e-9 * np.abs(want).max())


def test_gradient_antisymmetric_on_symmetric_lattice(orc):
    n = 11
    g = np.stack(np.meshgrid(*[np.arange(n)] * 3, indexing="ij"), -1).reshape(-1, 3) * 0.02
    P = np.concatenate([g, np.full((g.shape[0], 1), 0.07)], 1)
    rp, col = orc.neighbours(P)
    i = int(np.argmin(np.sum((g - g.mean(0)) ** 2, 1)))
    coef, status, _ = orc.stencils(P, np.zeros(len(P), np.uint8), rp, col, rows=[i])
    r = col[rp[i]:rp[i + 1]]
    off = np.round((g[r] - g[i]) / 0.02).astype(int)
    idx = {tuple(o): k for k, o in enumerate(off)}
    cf = coef[rp[i]:rp[i + 1]]
    for k, o in enumerate(off):
        m = idx[tuple(-o)]
        np.testing.assert_allclose(cf[k, :3], -cf[m, :3], atol=1e-9)
        assert abs(cf[k, 3] - cf[m, 3]) < 1e-6
    # Laplacian weights sum to zero (constant reproduced); centre weight negative
    assert abs(cf[:, 3].sum()) < 1e-7 and cf[list(r).index(i), 3] < 0


def test_rank_deficient_rows_are_zero(orc):
    # 3D particle with fewer than 10 same-model neighbours, and a planar 3D set
    P = np.array([[0, 0, 0, 1.0], [0.2, 0, 0, 1.0], [0, 0.2, 0, 1.0], [0, 0, 0.2, 1.0]])
    rp, col = orc.neighbours(P)
    coef, status, cond = orc.stencils(P, np.zeros(4, np.uint8), rp, col)
    assert np.all(status == 1) and np.all(coef == 0) and np.all(np.isinf(cond))
    f = C.flat_film(0.01, 0.2, 0.001, jitter=False)
    rp, col = orc.neighbours(f.pos_h)
    coef, status, cond = orc.stencils(f.pos_h, np.zeros(f.n, np.uint8), rp, col)
    assert np.all(status == 1)       # planar points cannot fix z-quadratics
    coef, status, cond = orc.stencils(f.pos_h, f.model, rp, col)
    assert np.all(status == 0)       # as a 2D model the same points are fine


def test_other_model_entries_are_zero(orc):
    c = C.config_small()
    rp, col = orc.neighbours(c.pos_h)
    coef, status, cond = orc.stencils(c.pos_h, c.model, rp, col)
    rows = np.repeat(np.arange(c.n), np.diff(rp))
    other = c.model[rows] != c.model[col]
    assert other.sum() > 0 and np.all(coef[other] == 0)


def test_apply_matches_scipy_and_transpose(orc):
    c = C.config_small()
    rp, col = orc.neighbours(c.pos_h)
    coef, status, cond = orc.stencils(c.pos_h, c.model, rp, col)
    out = orc.apply(rp, col, coef, c.vp)
    F = c.vp.astype(np.float64)
    for op in range(4):
        M = _csr(rp, col, coef[:, op], c.n)
        np.testing.assert_allclose(out[:, :, op], M @ F, rtol=1e-12, atol=1e-12)
    rng = np.random.default_rng(0)
    G = rng.normal(size=(c.n, 4, 4))
    gf = orc.apply_T(rp, col, coef, G)
    want = sum(_csr(rp, col, coef[:, op], c.n).T @ G[:, :, op] for op in range(4))
    np.testing.assert_allclose(gf, want, rtol=1e-10, atol=1e-10)
    # subset rows equal the full computation
    sub = orc.apply(rp, col, coef, c.vp, rows=[0, 17, 5000])
    np.testing.assert_array_equal(sub[[0, 17, 5000]], out[[0, 17, 5000]])


def test_pipeline_exact_on_quadratic_fields(orc):
    c = C.config_small()
    X = c.pos_h[:, :3].astype(np.float64)
    F = np.stack([X[:, 0] ** 2, X[:, 0] * X[:, 1], X[:, 2], 3 + X[:, 1]], 1)
    c.vp = F.astype(np.float32)
    rp, col = orc.neighbours(c.pos_h)
    coef, status, _ = orc.stencils(c.pos_h, c.model, rp, col)
    out = orc.apply(rp, col, coef, F)
    m3 = (c.model == 0)
    Xd = X
    np.testing.assert_allclose(out[m3, 0, 0], 2 * Xd[m3, 0], atol=1e-8)
    np.testing.assert_allclose(out[m3, 0, 3], 2.0, atol=1e-5)
    np.testing.assert_allclose(out[m3, 1, 0], Xd[m3, 1], atol=1e-8)
    np.testing.assert_allclose(out[m3, 1, 1], Xd[m3, 0], atol=1e-8)
    np.testing.assert_allclose(out[m3, 2, 2], 1.0, atol=1e-8)
    np.testing.assert_allclose(out[:, 3, 1], 1.0 * (c.model == 0) + 1.0 * (c.model == 1), atol=1e-8)
