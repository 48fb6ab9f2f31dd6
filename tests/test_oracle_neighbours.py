"""Pins of the oracle's neighbourhoods S_i (Eq. Nbd, Sec. 2.2)."""
import numpy as np
import pytest

from conftest import golden
from paper_2405_13165_gb300 import clouds as C


def test_hand_worked_rows(orc):
    P = np.array([[0, 0, 0, 0.5], [0.5, 0, 0, 0.5], [0, 0.75, 0, 1.0], [2, 2, 2, 0.25]])
    rp, col = orc.neighbours(P)
    for vals in golden("hand_worked.txt")["nbr_row"]:
        i = int(vals[0])
        want = [int(v) for v in vals[1:]]
        assert list(col[rp[i]:rp[i + 1]]) == want
        assert list(orc.row_brute(P, i)) == want


def test_bound_is_inclusive_and_tight(orc):
    # exactly at (h_i + h_j)/2 -> member; one float step beyond -> not a member
    P = np.array([[0, 0, 0, 0.5], [0.5, 0, 0, 0.5]])
    assert orc.in_support(P, 0, 1) and orc.in_support(P, 1, 0)
    P[1, 0] = np.nextafter(0.5, 1.0)
    assert not orc.in_support(P, 0, 1)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_cells_equal_brute_force(orc, seed):
    c = C.random_cloud(1500, seed=seed, h_lo=0.05, h_hi=0.2)
    rp, col = orc.neighbours(c.pos_h)
    for i in range(c.n):
        np.testing.assert_array_equal(col[rp[i]:rp[i + 1]], orc.row_brute(c.pos_h, i))


def test_cells_equal_numpy_distance_matrix(orc):
    # independent check: dense float64 distance matrix with the same rounding order
    c = C.random_cloud(700, seed=5)
    P = c.pos_h.astype(np.float64)
    d = P[None, :, :3] - P[:, None, :3]          # x_j - x_i
    d2 = (d[..., 0] * d[..., 0] + d[..., 1] * d[..., 1]) + d[..., 2] * d[..., 2]
    r = (P[:, None, 3] + P[None, :, 3]) * 0.5
    member = d2 <= r * r
    rp, col = orc.neighbours(c.pos_h)
    for i in range(c.n):
        np.testing.assert_array_equal(col[rp[i]:rp[i + 1]], np.nonzero(member[i])[0])


def test_self_member_symmetric_sorted(orc):
    c = C.config_small()
    rp, col = orc.neighbours(c.pos_h)
    rows = np.repeat(np.arange(c.n), np.diff(rp))
    pairs = set(zip(rows.tolist(), col.tolist()))
    assert all((i, i) in pairs for i in range(c.n))
    assert all((j, i) in pairs for (i, j) in pairs)
    for i in range(0, c.n, 97):
        r = col[rp[i]:rp[i + 1]]
        assert np.all(np.diff(r) > 0)


def test_degenerate_sizes(orc):
    rp, col = orc.neighbours(np.zeros((0, 4)))
    assert rp.tolist() == [0] and col.size == 0
    rp, col = orc.neighbours(np.array([[1.0, 2.0, 3.0, 0.1]]))
    assert rp.tolist() == [0, 1] and col.tolist() == [0]
    # coincident particles are all mutual neighbours
    P = np.tile(np.array([[0.3, 0.3, 0.3, 0.01]]), (5, 1))
    rp, col = orc.neighbours(P)
    assert np.all(np.diff(rp) == 5)


def test_lattice_count_matches_ball_volume(orc):
    # interior of an unjittered cubic lattice at h = 3.5 dx: |S_i| is the number
    # of integer points within radius 3.5, i.e. 179 (ball volume 179.6)
    c = C.cube_on_sheet(0.02)
    pts = np.stack(np.meshgrid(*[np.arange(-4, 5)] * 3, indexing="ij"), -1).reshape(-1, 3)
    want = int(np.sum(np.sum(pts * pts, 1) <= 3.5 ** 2))
    n = 11
    g = np.stack(np.meshgrid(*[np.arange(n)] * 3, indexing="ij"), -1).reshape(-1, 3) * 0.02
    P = np.concatenate([g, np.full((g.shape[0], 1), 0.07)], 1)
    rp, _ = orc.neighbours(P)
    centre = np.argmin(np.sum((g - g.mean(0)) ** 2, 1))
    assert rp[centre + 1] - rp[centre] == want == 179
    assert c.n == 5650
