"""Pins of the oracle's model transition (Sec. 5, Algs. 3 and 4)."""
import math

import numpy as np

from conftest import golden
from paper_2405_13165_gb300 import clouds as C


def _state(c):
    import oracle
    return oracle.cloud_state(c)


def _run(orc, c):
    rp, col = orc.neighbours(c.pos_h)
    cl = orc.classify(c.pos_h, c.model, c.ptype, c.normal, c.vol, c.h3d, c.user, rp, col)
    flag = orc.smooth(c.model, cl["preflag"], c.last, rp, col)
    return rp, col, flag


def test_hand_worked_3d_to_2d(orc):
    g = golden("hand_worked.txt")
    # wall particle 0 on the floor, interior particles 1 and 2 above it, a second
    # wall particle far away (so 1 and 2 are nearest to 0)
    P = np.array([[0, 0, 0, 1.0], [0, 0, 0.1, 1.0], [0, 0, 0.3, 1.0], [5, 5, 0, 1.0]])
    st = dict(pos_h=P, vp=np.array([[1, 0, 0, 0], [4, 0, 0, 0], [7, 0, 0, 0], [0, 0, 0, 0.]]),
              normal=np.tile([0, 0, 1.0, 0], (4, 1)), rho=np.full(4, 1000.0),
              eta=np.full(4, 1e-3), mass=np.array([1.0, 2.0, 3.0, 9.0]), diam=np.ones(4),
              hfilm=np.zeros(4), h3d=np.ones(4), model=np.zeros(4, np.uint8),
              ptype=np.array([2, 0, 0, 2], np.uint8), last=np.zeros(4, np.uint8))
    rp, col = orc.neighbours(P)
    out, o2n, n_out = orc.remap(st, np.array([1, 0, 0, 0], np.uint8), rp, col)
    assert n_out == 2 and o2n.tolist() == [0, -1, -1, 1]
    assert out["mass"][0] == float(g["remap_mass"][0][0])
    assert out["vp"][0, 0] == float(g["remap_u"][0][0])
    assert abs(out["hfilm"][0] - float(g["remap_H"][0][0])) < 1e-15
    assert out["model"][0] == 1 and out["last"][0] == 1 and out["last"][1] == 0
    # droplet diameter from m = rho V, V = pi d^3 / 6
    assert abs(math.pi * out["diam"][0] ** 3 / 6 * out["rho"][0] - out["mass"][0]) < 1e-12


def test_hand_worked_2d_to_3d(orc):
    g = golden("hand_worked.txt")
    P = np.array([[0, 0, 0, 0.35]])
    st = dict(pos_h=P, vp=np.array([[1, 2, 3, 4.0]]), normal=np.array([[0, 0, 1.0, 0]]),
              rho=np.array([1000.0]), eta=np.array([1e-3]), mass=np.array([8.0]),
              diam=np.ones(1), hfilm=np.array([0.25]), h3d=np.array([0.35]),
              model=np.ones(1, np.uint8), ptype=np.full(1, 2, np.uint8), last=np.zeros(1, np.uint8))
    rp, col = orc.neighbours(P)
    out, o2n, n_out = orc.remap(st, np.array([2], np.uint8), rp, col,
                                prm=dict(c_psi=1 / 3.5))
    gam = int(g["gamma_count"][0][0])
    assert n_out == 1 + gam
    np.testing.assert_allclose(out["mass"], 8.0 / (1 + gam))
    np.testing.assert_allclose(out["pos_h"][1:, 2], 0.25 / gam * np.arange(1, gam + 1), rtol=1e-15)
    assert out["ptype"].tolist() == [2] + [0] * (gam - 1) + [1]
    assert np.all(out["model"] == 0) and np.all(out["last"] == 1)
    np.testing.assert_array_equal(out["vp"], np.tile([1, 2, 3, 4.0], (1 + gam, 1)))


def test_shallow_cylinder_conserves_mass_and_volume(orc):
    # Sec. 7.1: mass and volume identical before and after, to rounding
    c = C.shallow_layer(dx=0.05, depth_layers=3, extent=1.0, cylinder=True, h_factor=6.0)
    rp, col, flag = _run(orc, c)
    out, o2n, n_out = orc.remap(_state(c), flag, rp, col)
    m_in = c.mass.astype(np.float64).sum()
    assert abs(out["mass"].sum() - m_in) <= 1e-12 * m_in
    v_in = (c.mass.astype(np.float64) / c.rho).sum()
    assert abs((out["mass"] / out["rho"]).sum() - v_in) <= 1e-12 * v_in
    # every floor particle is now a 2D film particle; interior all deleted near the floor
    assert (out["model"] == 1).sum() == (flag == 1).sum()
    assert np.all(out["last"][out["model"] == 1] == 1)


def test_deleted_particles_map_to_their_nearest_flagged_wall(orc):
    c = C.shallow_layer(dx=0.05, depth_layers=3, extent=0.8, cylinder=True, h_factor=6.0,
                        seed=3)
    rp, col, flag = _run(orc, c)
    out, o2n, n_out = orc.remap(_state(c), flag, rp, col)
    P = c.pos_h.astype(np.float64)
    wall = np.nonzero((c.ptype == 2) & (c.model == 0))[0]
    cand = np.zeros(c.n, bool)
    for i in np.nonzero(flag == 1)[0]:
        r = col[rp[i]:rp[i + 1]]
        cand[r[(c.ptype[r] != 2) & (c.model[r] == 0)]] = True
    for b in range(c.n):
        r = set(col[rp[b]:rp[b + 1]].tolist())
        ws = [w for w in wall if w in r]
        if not cand[b] or not ws:
            assert o2n[b] >= 0
            continue
        d2 = [np.sum((P[w, :3] - P[b, :3]) ** 2) for w in ws]
        jw = ws[int(np.argmin(d2))]
        assert (o2n[b] < 0) == (flag[jw] == 1)


def test_depth_constant_field_is_unchanged(orc):
    # Sec. 7.2: data transfer exact for fields constant along the depth
    c = C.shallow_layer(dx=0.05, depth_layers=3, extent=1.0, cylinder=True, h_factor=6.0)
    c.vp[:, 0] = np.sin(3 * c.pos_h[:, 0]) + c.pos_h[:, 1]
    rp, col, flag = _run(orc, c)
    out, o2n, n_out = orc.remap(_state(c), flag, rp, col)
    # a 2D particle that absorbed particles straight above it (no jitter in x,y
    # along the column) keeps the column's value exactly
    c2 = C.shallow_layer(dx=0.05, depth_layers=3, extent=1.0, cylinder=True, h_factor=6.0,
                         jitter=False)
    c2.vp[:, 3] = np.cos(2 * c2.pos_h[:, 0]) * np.sin(c2.pos_h[:, 1])
    rp2, col2, flag2 = _run(orc, c2)
    out2, o2n2, _ = orc.remap(_state(c2), flag2, rp2, col2)
    assert n_out > 0
    moved = np.nonzero(flag2 == 1)[0]
    for i in moved[:200]:
        absorbed = [b for b in col2[rp2[i]:rp2[i + 1]] if o2n2[b] < 0 and
                    abs(c2.pos_h[b, 0] - c2.pos_h[i, 0]) < 1e-12 and
                    abs(c2.pos_h[b, 1] - c2.pos_h[i, 1]) < 1e-12]
        cnt = sum(1 for b in col2[rp2[i]:rp2[i + 1]] if o2n2[b] < 0 and
                  c2.pos_h[b, 2] > 0)
        if cnt == len(absorbed):
            assert abs(out2["vp"][o2n2[i], 3] - float(c2.vp[i, 3])) < 1e-6


def test_round_trip_2d_3d_2d(orc):
    # a film column lifted to 3D and collapsed again keeps its mass exactly and
    # its height within one spacing psi
    f = C.flat_film(0.01, 0.2, 0.004, jitter=False)
    st = _state(f)
    st["hfilm"] = np.full(f.n, 0.02)
    rp, col = orc.neighbours(f.pos_h)
    out, o2n, n_out = orc.remap(st, np.full(f.n, 2, np.uint8), rp, col)
    gamma = math.ceil(0.02 / (orc.DEFAULT_PARAMS["c_psi"] * float(f.h3d[0])))
    assert n_out == f.n * (1 + gamma)
    m0 = f.mass.astype(np.float64).sum()
    assert abs(out["mass"].sum() - m0) <= 1e-12 * m0
    rp2, col2 = orc.neighbours(out["pos_h"])
    flag = np.where((out["ptype"] == 2), 1, 0).astype(np.uint8)
    back, o2n2, n_back = orc.remap(out, flag, rp2, col2)
    assert n_back == f.n
    assert abs(back["mass"].sum() - m0) <= 1e-12 * m0
    psi = 0.02 / gamma
    assert np.all(np.abs(back["hfilm"] - 0.02) <= psi + 1e-12)


def test_candidates_from_flagged_rows_equal_the_definition(orc):
    """Alg. 3's candidates (interior / free-surface 3D particles b with a 3D
    particle flagged 3D -> 2D in S_b) are the same set when read from the rows
    of the flagged particles, because S is symmetric (Eq. Nbd): the GPU remap
    marks them that way.  Checked on the shallow cylinder (flagged floor) and
    on a random cloud with variable h and an arbitrary flag set."""
    clouds = [C.shallow_layer(dx=0.05, depth_layers=3, extent=1.0, cylinder=True, h_factor=6.0)]
    rc = C.random_cloud(2000, seed=5, h_lo=0.05, h_hi=0.2)
    clouds.append(rc)
    for k, c in enumerate(clouds):
        if k == 0:
            rp, col, flag = _run(orc, c)
        else:
            rp, col = orc.neighbours(c.pos_h)
            rng = np.random.default_rng(9)
            flag = np.where(rng.random(c.n) < 0.05, 1, 0).astype(np.uint8)
            c.model[:] = np.where(rng.random(c.n) < 0.8, 0, 1).astype(np.uint8)
            c.ptype[:] = rng.integers(0, 3, c.n).astype(np.uint8)
        is3 = c.model == 0
        inner = is3 & (c.ptype != C.TYPE_WALL)
        flagged = is3 & (flag == 1)
        by_def = np.zeros(c.n, bool)
        for b in np.nonzero(inner)[0]:
            by_def[b] = flagged[col[rp[b]:rp[b + 1]]].any()
        by_rows = np.zeros(c.n, bool)
        for j in np.nonzero(flagged)[0]:
            nb = col[rp[j]:rp[j + 1]]
            by_rows[nb[inner[nb]]] = True
        assert by_def.any()
        np.testing.assert_array_equal(by_rows, by_def)
