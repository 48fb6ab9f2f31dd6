"""Pins of the film momentum step (Eq. FilmMomentum) and the post-processing
quantities (Eq. InstFlux; n^T S n) of the oracle."""
import numpy as np

from paper_2405_13165_gb300 import clouds as C


def test_film_momentum_closed_forms(orc):
    n = 4
    model = np.array([1, 1, 1, 0], np.uint8)
    vp = np.array([[1.0, 2.0, 0.0, 5.0]] * n)
    rho = np.full(n, 1000.0)
    eta = np.full(n, 1e-3)
    H = np.array([1e-3, 1e-3, 0.0, 1e-3])
    normal = np.tile([0.0, 0.0, 1.0, 0.0], (n, 1))
    out = np.zeros((n, 4, 4))
    dt = 0.01
    # pure damping: v (1 - dt eta / (rho H^2))
    new = orc.film_momentum(model, vp, rho, eta, H, normal, out, [0, 0, 0], dt)
    f = 1.0 - dt * 1e-3 / (1000.0 * 1e-6)
    np.testing.assert_allclose(new[0, :3], [f * 1.0, f * 2.0, 0.0], rtol=1e-15)
    np.testing.assert_array_equal(new[2], vp[2])          # H = 0: untouched
    np.testing.assert_array_equal(new[3], vp[3])          # 3D: untouched
    assert new[0, 3] == 5.0                               # pressure slot kept
    # gravity along a tilted plate: only its tangential part acts, result tangential
    nt = np.array([0.0, np.sin(0.3), np.cos(0.3)])
    normal2 = np.tile(np.append(nt, 0.0), (n, 1))
    v0 = np.zeros((n, 4))
    new = orc.film_momentum(model, v0, rho, np.zeros(n), H, normal2, out, [0, 0, -9.81], dt)
    g = np.array([0, 0, -9.81])
    gpar = g - (g @ nt) * nt
    np.testing.assert_allclose(new[0, :3], dt * gpar, rtol=1e-14)
    assert abs(new[0, :3] @ nt) < 1e-15
    # pressure gradient: -dt grad p / rho
    out2 = np.zeros((n, 4, 4))
    out2[:, 3, :3] = [100.0, -50.0, 0.0]
    new = orc.film_momentum(model, v0, rho, np.zeros(n), H, normal, out2, [0, 0, 0], dt)
    np.testing.assert_allclose(new[0, :3], [-dt * 0.1, dt * 0.05, 0.0], rtol=1e-14)


def test_plane_flux_counts_crossings(orc):
    rng = np.random.default_rng(3)
    p0 = np.zeros((6, 4))
    p0[:, 0] = [-0.1, -0.2, 0.3, 0.05, -0.01, 0.2]
    p1 = p0.copy()
    p1[:, 0] = [0.1, -0.1, -0.3, 0.06, 0.0, 0.25]
    mass = rng.uniform(1, 2, 6)
    rho = np.full(6, 1000.0)
    vol, cnt = orc.plane_flux(p0, p1, mass, rho, [0, 0, 0], [1, 0, 0])
    v = mass / rho
    assert cnt == 3                       # particles 0 and 4 forward, 2 back
    assert abs(vol - (v[0] + v[4] - v[2])) < 1e-18


def test_normal_stress_of_linear_fields_is_exact(orc):
    # stencils differentiate linear velocity fields exactly, so n^T S n of
    # v = G x is 2 eta n^T G n at every regular 3D particle
    c = C.cube_on_sheet(0.05, cube=0.4, sheet=1.0)
    P = c.pos_h.astype(np.float64)
    G = np.array([[0.3, -1.0, 0.5], [2.0, 0.1, -0.4], [0.7, 1.5, -0.2]])
    F = np.zeros((c.n, 4))
    F[:, :3] = P[:, :3] @ G.T
    rp, col = orc.neighbours(P)
    coef, status, _ = orc.stencils(P, c.model, rp, col)
    out = orc.apply(rp, col, coef, F)
    sel = ((c.model == 0) & (status == 0)).astype(np.uint8)
    normal = np.tile([0.0, 0.0, 1.0, 0.0], (c.n, 1))
    s, cnt = orc.normal_stress(sel, out, c.eta, normal)
    want = 2.0 * c.eta.astype(np.float64)[sel.astype(bool)] * G[2, 2]
    assert cnt == sel.sum() > 0
    assert abs(s - want.sum()) <= 1e-9 * abs(want.sum())
