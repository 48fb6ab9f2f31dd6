"""Pins of the oracle's position gradient through the GFDM stencils against
central finite differences in FP64 (neighbour sets held fixed), on flat,
tilted and curved films, every coordinate of the film particles included."""
import numpy as np
import pytest

from paper_2405_13165_gb300 import clouds as C
from grad_shapes import SHAPES, shape as _shape


def _loss(orc, P, model, rp, col, F, G):
    coef, status, _ = orc.stencils(P, model, rp, col)
    out = orc.apply(rp, col, coef, F)
    return float(np.sum(out * G)), out


def _safe_coords(P, rp, col, i, step):
    """Coordinate i is usable when no pair involving it sits within 10 steps
    of the support boundary (W' jumps there)."""
    r = col[rp[i]:rp[i + 1]]
    d = np.linalg.norm(P[r, :3] - P[i, :3], axis=1)
    return np.all(np.abs(d - P[i, 3]) > 10 * step)


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("loss", ["laplacian", "random"])
def test_gradient_matches_central_differences(orc, loss, shape):
    c, dx = _shape(shape)
    P = c.pos_h.astype(np.float64)
    F = c.vp.astype(np.float64)
    rp, col = orc.neighbours(P)
    rng = np.random.default_rng(1)
    coef, status, _ = orc.stencils(P, c.model, rp, col)
    out = orc.apply(rp, col, coef, F)
    if loss == "laplacian":
        # L = sum_i sum_f (Lap_i f)^2  ->  dL/dout = 2 Lap on the Laplacian channel
        G = np.zeros_like(out)
        G[:, :, 3] = 2.0 * out[:, :, 3]
    else:
        G = rng.normal(size=out.shape)
    g = orc.stencil_grad(P, c.model, rp, col, F, G)
    step = 1e-4 * dx
    # film particles first: every coordinate of theirs moves the PCA frame of
    # the film rows around them
    film = np.nonzero(c.model == 1)[0]
    bulk = np.nonzero(c.model == 0)[0]
    picks = np.concatenate([rng.choice(film, 40, replace=False),
                            rng.choice(bulk, min(20, bulk.size), replace=False)])
    checked = film_z = 0
    for i in picks:
        if not _safe_coords(P, rp, col, i, step):
            continue
        for a in (0, 1, 2):
            def central(st):
                Pp = P.copy()
                Pm = P.copy()
                Pp[i, a] += st
                Pm[i, a] -= st
                if loss == "laplacian":
                    lp = np.sum(_loss(orc, Pp, c.model, rp, col, F, G)[1][:, :, 3] ** 2)
                    lm = np.sum(_loss(orc, Pm, c.model, rp, col, F, G)[1][:, :, 3] ** 2)
                else:
                    lp = _loss(orc, Pp, c.model, rp, col, F, G)[0]
                    lm = _loss(orc, Pm, c.model, rp, col, F, G)[0]
                return (lp - lm) / (2 * st)
            # Richardson: the O(step^2) error of the central difference cancels
            fd = (4.0 * central(step / 2) - central(step)) / 3.0
            scale = max(abs(fd), 1e-3 * np.abs(g[:, :3]).max())
            assert abs(g[i, a] - fd) <= 2e-5 * scale + 1e-9, (shape, i, a, g[i, a], fd)
            checked += 1
            film_z += int(c.model[i] == 1 and a == 2)
    assert checked >= 120 and film_z >= 30
    assert np.all(g[:, 3] == 0.0)


def test_film_frame_term_is_what_moves_a_flat_film_out_of_plane(orc):
    # On a flat film every neighbour lies in the tangent plane, so moving a film
    # particle out of the plane changes no in-plane coordinate and no weight to
    # first order: its z-gradient comes only from the PCA normal turning the
    # world-coordinate gradient outputs.  A loss on the Laplacian alone does
    # not see that turn (the plane Laplacian ignores the frame's orientation),
    # a loss on the gradient outputs does.
    c = C.flat_film(0.05, 0.8, 0.015)
    P = c.pos_h.astype(np.float64)
    F = c.vp.astype(np.float64)
    rp, col = orc.neighbours(P)
    rng = np.random.default_rng(4)
    G = rng.normal(size=(c.n, 4, 4))
    G_lap = G.copy()
    G_lap[:, :, :3] = 0.0
    G_grad = G.copy()
    G_grad[:, :, 3] = 0.0
    assert np.all(orc.stencil_grad(P, c.model, rp, col, F, G_lap)[:, 2] == 0.0)
    gz = orc.stencil_grad(P, c.model, rp, col, F, G_grad)[:, 2]
    assert np.abs(gz).max() > 0.1 * np.abs(orc.stencil_grad(P, c.model, rp, col, F, G_grad)[:, :2]).max()


def test_gradient_of_translation_invariant_loss_sums_to_zero(orc):
    # stencils depend on differences x_j - x_i only, so translating every
    # particle changes nothing: the gradient summed over particles vanishes
    c = C.cube_on_sheet(0.05, cube=0.4, sheet=1.0)
    P = c.pos_h.astype(np.float64)
    rp, col = orc.neighbours(P)
    rng = np.random.default_rng(2)
    G = rng.normal(size=(c.n, 4, 4))
    # fields moving with the particles (u_j - u_i fixed): only the stencils change
    g = orc.stencil_grad(P, c.model, rp, col, c.vp.astype(np.float64), G)
    tot = g[:, :3].sum(0)
    assert np.all(np.abs(tot) <= 1e-9 * np.abs(g[:, :3]).sum(0))


def test_gradient_zero_for_deficient_rows(orc):
    P = np.array([[0, 0, 0, 1.0], [0.2, 0, 0, 1.0], [0, 0.2, 0, 1.0], [0, 0, 0.2, 1.0]])
    rp, col = orc.neighbours(P)
    g = orc.stencil_grad(P, np.zeros(4, np.uint8), rp, col, np.ones((4, 4)),
                         np.ones((4, 4, 4)))
    assert np.all(g == 0)


def test_gradient_is_additive_over_rows(orc):
    # the gradient is linear in dL/dout, so splitting the rows into two sets and
    # adding the two gradients gives the full one (also covers rows whose output
    # gradient is zero, which contribute nothing)
    c = C.cube_on_sheet(0.05, cube=0.4, sheet=1.0)
    P = c.pos_h.astype(np.float64)
    F = c.vp.astype(np.float64)
    rp, col = orc.neighbours(P)
    rng = np.random.default_rng(7)
    G = rng.normal(size=(c.n, 4, 4))
    part = rng.uniform(size=c.n) < 0.3
    Ga, Gb = G.copy(), G.copy()
    Ga[~part] = 0.0
    Gb[part] = 0.0
    g = orc.stencil_grad(P, c.model, rp, col, F, G)
    ga = orc.stencil_grad(P, c.model, rp, col, F, Ga)
    gb = orc.stencil_grad(P, c.model, rp, col, F, Gb)
    assert np.all(np.abs(ga + gb - g) <= 1e-12 * np.abs(g).max())
    assert np.any(ga[:, :3] != 0) and np.any(gb[:, :3] != 0)
