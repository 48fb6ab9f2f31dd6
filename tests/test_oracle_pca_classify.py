"""Pins of the oracle's detection stage: local PCA (Sec. 4.1.2), eigenvector test
(Sec. 4.1.3), Alg. 2, film height (Eq. Height), Eq. 2Dto3Dcond and smoothing
(Sec. 4.3)."""
import math

import numpy as np
import pytest

from conftest import golden
from paper_2405_13165_gb300 import clouds as C


def _params():
    g = golden("paper_constants.txt")
    return float(g["eps_lambda_max"][0][0]), float(g["theta_star_over_pi"][0][0]) * math.pi


def test_default_params_are_the_papers(orc):
    eps, th = _params()
    assert orc.DEFAULT_PARAMS["eps_lambda_max"] == eps
    assert abs(orc.DEFAULT_PARAMS["theta_star"] - th) < 1e-15


@pytest.mark.parametrize("seed", range(5))
def test_jacobi_matches_eigh(orc, seed):
    rng = np.random.default_rng(seed)
    B = rng.normal(size=(3, 3))
    A = B @ B.T if seed % 2 else B + B.T
    lam, V = orc.jacobi3(A)
    w, U = np.linalg.eigh(A)
    np.testing.assert_allclose(lam, w[::-1], rtol=1e-12, atol=1e-12 * np.abs(w).max())
    for k in range(3):
        assert abs(abs(V[:, k] @ U[:, 2 - k]) - 1.0) < 1e-10
    np.testing.assert_allclose(V @ np.diag(lam) @ V.T, A, atol=1e-12 * np.abs(A).max())


def test_jacobi_degenerate_and_diagonal(orc):
    lam, V = orc.jacobi3(np.diag([2.0, 5.0, 5.0]))
    np.testing.assert_allclose(lam, [5, 5, 2])
    lam, V = orc.jacobi3(np.zeros((3, 3)))
    np.testing.assert_allclose(lam, [0, 0, 0])
    np.testing.assert_allclose(np.abs(V.T @ V), np.eye(3), atol=1e-15)


def test_hand_worked_square(orc):
    g = golden("hand_worked.txt")
    P = np.array([[0, 0, 0, 1.0], [1, 0, 0, 1.0], [0, 1, 0, 1.0], [1, 1, 0, 1.0]])
    rp = np.array([0, 4, 8, 12, 16])
    col = np.tile(np.arange(4, dtype=np.int32), 4)
    m, lam, V = orc.pca(P, np.zeros(4, np.uint8), rp, col, 0)
    assert m == 4
    np.testing.assert_allclose(lam, [float(v) for v in g["pca_lambda"][0]], atol=1e-15)
    assert abs(abs(V[2, 2]) - 1.0) < 1e-15


def test_pca_equals_scatter_matrix(orc):
    # P_i = sum (x_j - x_c)(x_j - x_c)^T equals n * (biased covariance) of q = (x-x_i)/h
    c = C.random_cloud(600, seed=3, frac2d=0.0)
    rp, col = orc.neighbours(c.pos_h)
    for i in [5, 50, 300]:
        r = col[rp[i]:rp[i + 1]]
        q = (c.pos_h[r, :3].astype(float) - c.pos_h[i, :3].astype(float)) / float(c.pos_h[i, 3])
        S = np.cov(q.T, bias=True) * len(r)
        m, lam, V = orc.pca(c.pos_h, c.model, rp, col, i)
        np.testing.assert_allclose(lam, np.linalg.eigvalsh(S)[::-1], rtol=1e-10, atol=1e-14)


def test_planar_and_collinear_sets(orc):
    f = C.flat_film(0.01, 0.3, 0.001)
    rp, col = orc.neighbours(f.pos_h)
    cl = orc.classify(f.pos_h, f.model, f.ptype, f.normal, f.vol, f.h3d, f.user, rp, col)
    assert np.all(cl["eig"][:, 2] == 0.0) and np.all(cl["eig"][:, 3] == 0.0)
    assert np.all(np.abs(np.abs(cl["frame"][:, 6]) - 1.0) < 1e-15)  # w3 = +-z
    # collinear points: two vanishing eigenvalues
    P = np.zeros((9, 4))
    P[:, 0] = np.arange(9) * 0.1
    P[:, 3] = 0.5
    rp, col = orc.neighbours(P)
    m, lam, V = orc.pca(P, np.zeros(9, np.uint8), rp, col, 4)
    assert lam[0] > 0 and abs(lam[1]) < 1e-15 * lam[0] and abs(lam[2]) < 1e-15 * lam[0]
    assert abs(abs(V[0, 0]) - 1) < 1e-12


def test_isotropic_lattice_is_bulk(orc):
    n = 11
    g = np.stack(np.meshgrid(*[np.arange(n)] * 3, indexing="ij"), -1).reshape(-1, 3) * 0.02
    P = np.concatenate([g, np.full((g.shape[0], 1), 0.07)], 1)
    rp, col = orc.neighbours(P)
    i = np.argmin(np.sum((g - g.mean(0)) ** 2, 1))
    m, lam, V = orc.pca(P, np.zeros(len(P), np.uint8), rp, col, i)
    np.testing.assert_allclose(lam, lam[0], rtol=1e-12)  # cubic symmetry: P = c I


def _shallow(h_factor):
    return C.shallow_layer(dx=0.05, depth_layers=3, extent=1.0, cylinder=True, h_factor=h_factor)


def test_shallow_cylinder_floor_transitions_side_walls_do_not(orc):
    # Sec. 7.1: after coarsening, every floor wall particle transitions to 2D,
    # while side-wall particles fail the eigenvector test.  This fixes the
    # direction of Eq. EigenvectorLimit.
    c = _shallow(6.0)
    rp, col = orc.neighbours(c.pos_h)
    cl = orc.classify(c.pos_h, c.model, c.ptype, c.normal, c.vol, c.h3d, c.user, rp, col)
    side = (c.ptype == C.TYPE_WALL) & (np.abs(c.normal[:, 2]) < 0.5)
    floor = (c.ptype == C.TYPE_WALL) & ~side
    assert np.all(cl["preflag"][floor] == 1)
    assert np.all(cl["preflag"][side] == 0)
    assert np.all(cl["preflag"][c.ptype != C.TYPE_WALL] == 0)
    flag = orc.smooth(c.model, cl["preflag"], c.last, rp, col)
    np.testing.assert_array_equal(flag, cl["preflag"])   # all at once (Sec. 7.1)


def test_fine_resolution_keeps_3d(orc):
    # deep layer resolved by h: wall particles see interior but no free-surface
    # neighbours -> resolution criterion says stay 3D
    c = C.shallow_layer(dx=0.05, depth_layers=8, extent=0.6, cylinder=False, h_factor=3.5)
    rp, col = orc.neighbours(c.pos_h)
    cl = orc.classify(c.pos_h, c.model, c.ptype, c.normal, c.vol, c.h3d, c.user, rp, col)
    floor = (c.ptype == C.TYPE_WALL) & (c.normal[:, 2] > 0.5)
    assert np.all(cl["preflag"][floor] == 0)


def test_resolution_criterion_branches(orc):
    # particle 0: 3D wall at origin; neighbours chosen by hand
    base = np.array([[0, 0, 0, 1.0], [0.3, 0, 0, 1.0], [0, 0.3, 0, 1.0], [0, 0, 0.3, 1.0]])
    model = np.zeros(4, np.uint8)
    normal = np.zeros((4, 4))
    normal[:, 2] = 1
    rp, col = orc.neighbours(base)
    vol = np.ones(4)
    h3d = np.ones(4)

    def pre(types, user=0):
        u = np.zeros(4, np.uint8)
        u[0] = user
        return orc.classify(base, model, np.array(types, np.uint8), normal, vol, h3d, u,
                            rp, col)["preflag"][0]
    W, I, F = C.TYPE_WALL, C.TYPE_INTERIOR, C.TYPE_FREE_SURFACE
    assert pre([W, W, W, W]) == 1                     # only wall neighbours
    assert pre([W, I, W, W]) == 0                     # interior, no free surface
    assert pre([W, I, W, W], user=C.USER_TO_2D) == 0  # user flag inside resolution branch
    # free surface present -> PCA: 3 orthogonal unit offsets + origin is 3D-ish
    assert pre([W, F, W, W]) == 0
    assert pre([W, F, W, W], user=C.USER_TO_2D) == 1
    # make the neighbourhood planar (z = 0) with normal +z -> eps = 0, |n.w3| = 1
    flat = base.copy()
    flat[3] = [0.2, 0.2, 0, 1.0]
    rp2, col2 = orc.neighbours(flat)
    t = np.array([W, F, W, W], np.uint8)
    got = orc.classify(flat, model, t, normal, vol, h3d, np.zeros(4, np.uint8), rp2, col2)
    assert got["preflag"][0] == 1 and got["eig"][0, 3] < 1e-12
    # same plane, wall normal in the plane (n.w3 = 0): eigenvector test fails
    n2 = normal.copy()
    n2[:, :3] = [1, 0, 0]
    got = orc.classify(flat, model, t, n2, vol, h3d, np.zeros(4, np.uint8), rp2, col2)
    assert got["preflag"][0] == 0


def test_eigenvector_angle_threshold(orc):
    # planar neighbourhood, normal tilted by angle a from w3 = z: flagged iff a <= pi/6
    flat = np.array([[0, 0, 0, 1.0], [0.3, 0, 0, 1.0], [0, 0.3, 0, 1.0], [0.2, 0.2, 0, 1.0]])
    model = np.zeros(4, np.uint8)
    t = np.array([2, 1, 2, 2], np.uint8)
    rp, col = orc.neighbours(flat)
    for a, want in [(0.0, 1), (0.5, 1), (math.pi / 6 - 1e-3, 1), (math.pi / 6 + 1e-3, 0),
                    (1.2, 0)]:
        nrm = np.zeros((4, 4))
        nrm[:, 0] = math.sin(a)
        nrm[:, 2] = math.cos(a)
        got = orc.classify(flat, model, t, nrm, np.ones(4), np.ones(4), np.zeros(4, np.uint8),
                           rp, col)
        assert got["preflag"][0] == want, a


def test_hfilm_hand_worked(orc):
    g = golden("hand_worked.txt")
    P = np.array([[0, 0, 0, 1.0], [0.5, 0, 0, 1.0]])
    rp, col = orc.neighbours(P)
    cl = orc.classify(P, np.ones(2, np.uint8), np.full(2, 2, np.uint8), np.zeros((2, 4)),
                      np.full(2, 2.0), np.full(2, 100.0), np.zeros(2, np.uint8), rp, col)
    assert abs(cl["hfilm"][0] - float(g["hfilm_two"][0][0])) < 1e-14


@pytest.mark.parametrize("hf,tol", [(3.5, 4e-3), (16.0, 1.5e-3)])
def test_hfilm_closed_form_on_lattice(orc, hf, tol):
    # uniform film of volume V per particle on a square lattice: the kernel of
    # Eq. Height integrates to 1 - exp(-alpha) over the support, so H -> V/dx^2 (1-e^-alpha)
    dx, Hf = 0.01, 0.003
    f = C.flat_film(dx, 1.0, Hf, jitter=False, h_factor=hf)
    rp, col = orc.neighbours(f.pos_h)
    i = int(np.argmin(np.sum((f.pos_h[:, :2] - 0.5) ** 2, 1)))
    cl = orc.classify(f.pos_h, f.model, f.ptype, f.normal, f.vol, f.h3d, f.user, rp, col,
                      rows=[i])
    want = float(f.vol[0]) / dx ** 2 * (1 - math.exp(-orc.DEFAULT_PARAMS["alpha_film"]))
    assert abs(cl["hfilm"][i] / want - 1) < tol


def test_film_to_bulk_condition(orc):
    f = C.flat_film(0.01, 0.4, 0.003, jitter=False)
    rp, col = orc.neighbours(f.pos_h)
    h3d = f.h3d.copy()
    cl = orc.classify(f.pos_h, f.model, f.ptype, f.normal, f.vol, h3d, f.user, rp, col)
    assert np.all(cl["preflag"] == 0)            # H << h3D
    h3d[:] = 0.5 * cl["hfilm"].min()
    cl = orc.classify(f.pos_h, f.model, f.ptype, f.normal, f.vol, h3d, f.user, rp, col)
    assert np.all(cl["preflag"] == 2)            # H >= h3D everywhere
    u = f.user.copy()
    u[7] = C.USER_TO_3D
    cl = orc.classify(f.pos_h, f.model, f.ptype, f.normal, f.vol, f.h3d, u, rp, col)
    assert cl["preflag"][7] == 2 and cl["preflag"].sum() == 2


def test_smoothing_rules(orc):
    # chain of five 3D particles 0..4 on a line, spacing 1, h = 1.5 (neighbours +-1)
    P = np.zeros((5, 4))
    P[:, 0] = np.arange(5)
    P[:, 3] = 1.5
    rp, col = orc.neighbours(P)
    model = np.zeros(5, np.uint8)
    last = np.zeros(5, np.uint8)
    pre = np.array([0, 0, 1, 0, 0], np.uint8)
    # rule 1: lone flagged particle, no 2D neighbour -> not transitioned
    assert orc.smooth(model, pre, last, rp, col).tolist() == [0] * 5
    # a 2D neighbour exists -> kept
    m2 = model.copy()
    m2[3] = 1
    assert orc.smooth(m2, pre, last, rp, col).tolist() == [0, 0, 1, 0, 0]
    # a neighbour flagged for the same target -> both kept
    pre2 = np.array([0, 1, 1, 0, 0], np.uint8)
    assert orc.smooth(model, pre2, last, rp, col).tolist() == [0, 1, 1, 0, 0]
    # rule 2: transitioned in the previous step -> not transitioned again
    l2 = last.copy()
    l2[2] = 1
    assert orc.smooth(model, pre2, l2, rp, col).tolist() == [0, 1, 0, 0, 0]
