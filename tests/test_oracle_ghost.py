"""Pins of the oracle's buffer zone (Sec. 5.3, Alg. 5)."""
import numpy as np

from paper_2405_13165_gb300 import clouds as C


def test_ghost_sources_brute_force(orc):
    c = C.random_cloud(400, seed=3, h_lo=0.1, h_hi=0.2, frac2d=0.5)
    P = c.pos_h.astype(np.float64)
    rp, col = orc.neighbours(P)
    src = orc.ghost_sources(c.model, rp, col)
    d = np.linalg.norm(P[:, None, :3] - P[None, :, :3], axis=2)
    r = 0.5 * (P[:, None, 3] + P[None, :, 3])
    other = c.model[:, None] != c.model[None, :]
    want = np.any((d <= r) & other, axis=1)
    np.testing.assert_array_equal(src.astype(bool), want)
    assert 0 < src.sum() < c.n


def _zone(orc, c):
    st = orc.cloud_state(c)
    rp, col = orc.neighbours(c.pos_h)
    return orc.ghost_zone(st, rp, col), rp, col


def test_ghosts_transition_and_conserve_mass(orc):
    c = C.interface_strip(quadratic=True)
    (u, src, gflag, ng), rp, col = _zone(orc, c)
    n = c.n
    idx = np.nonzero(src)[0]
    # intermediate ghosts: one per source; flags follow model and type
    assert ng == idx.size
    np.testing.assert_array_equal(gflag == 2, c.model[idx] == 1)
    np.testing.assert_array_equal(gflag == 1, (c.model[idx] == 0) & (c.ptype[idx] == 2))
    gm = u["model"][n:]
    src3 = idx[c.model[idx] == 0]
    src2 = idx[c.model[idx] == 1]
    # 2D sources became 3D columns (walls at the film places plus gamma above),
    # 3D walls became film particles; every interior / free-surface 3D ghost was
    # mapped onto a wall ghost here, so the ghosts carry exactly the sources' mass
    assert (gm == 1).sum() == (gflag == 1).sum()
    assert (gm == 0).sum() == src2.size * 2 + src2.size       # gamma = 2 (H = 2 dx, psi~ = dx)
    m_src = c.mass[idx].astype(np.float64).sum()
    m_gh = u["mass"][n:].astype(np.float64).sum()
    assert abs(m_gh - m_src) <= 1e-6 * m_src
    assert abs(u["mass"][n:][gm == 0].astype(np.float64).sum()
               - c.mass[src2].astype(np.float64).sum()) <= 1e-6 * m_src
    # the regular particles are untouched and come first
    np.testing.assert_array_equal(u["pos_h"][:n], c.pos_h)
    # 3D ghosts lie over the film sources (x, y of a source), 2D ghosts at wall sources
    P = u["pos_h"][n:]
    fx = {tuple(np.round(p[:2], 6)) for p in c.pos_h[src2]}
    assert all(tuple(np.round(p[:2], 6)) in fx for p in P[gm == 0])


def test_quadratic_fields_exact_with_ghosts_and_coupled(orc):
    # depth-constant quadratic fields on vertical columns: the ghosts carry
    # exact samples (copies for film -> 3D, column averages for 3D -> film), so
    # derivatives at regular particles next to the buffer zone stay exact; and
    # a regular 3D particle next to the interface sees film data through its
    # 3D ghosts
    c = C.interface_strip(quadratic=True, columns=True)
    (u, src, gflag, ng), rp0, col0 = _zone(orc, c)
    n = c.n
    P = u["pos_h"].astype(np.float64)
    rp, col = orc.neighbours(P)
    rows = np.arange(n)
    coef, status, _ = orc.stencils(P, u["model"], rp, col, rows=rows)
    out = orc.apply(rp, col, coef, u["vp"], rows=rows)
    X, Y = P[:n, 0], P[:n, 1]
    Q = C.QUAD_FIELDS
    gx = Q[:, 1][None, :] + 2 * Q[:, 3][None, :] * X[:, None] + Q[:, 4][None, :] * Y[:, None]
    gy = Q[:, 2][None, :] + Q[:, 4][None, :] * X[:, None] + 2 * Q[:, 5][None, :] * Y[:, None]
    lap = np.broadcast_to(2 * Q[:, 3] + 2 * Q[:, 5], gx.shape)
    ok = status[:n] == 0
    near = src.astype(bool) & ok
    assert near.sum() > 100
    # exact up to the FP32 rounding of the stored field samples, which a stencil
    # can amplify by sum_j |c_ij| |u_j| * 2^-23 (a wrong ghost value would be
    # off by ~1e-2)
    bound = orc.apply(rp, col, np.abs(coef), np.abs(u["vp"]), rows=rows)[:n] * 2.0 ** -23
    for k, want in ((0, gx), (1, gy), (3, lap)):
        err = np.abs(out[:n, :, k][near] - want[near])
        allow = 2.0 * bound[:, :, k][near] + 1e-9 * np.abs(want).max()
        assert np.all(err <= allow), (k, (err / allow).max())
    # coupling: change the film data the ghosts were made from
    j = np.nonzero(src.astype(bool) & (c.model == 1))[0][0]
    c2 = C.interface_strip(quadratic=True, columns=True)
    c2.vp[j] += 1.0
    (u2, *_), _, _ = _zone(orc, c2)
    out2 = orc.apply(rp, col, coef, u2["vp"], rows=rows)
    moved = np.abs(out2[:n] - out[:n]).max(axis=(1, 2)) > 0
    assert np.any(moved & (c.model == 0)), "no regular 3D particle saw the film change"
