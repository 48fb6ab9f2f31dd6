"""Host-side pieces of the tray loop: the torch loop's advection and user
criterion agree bit for bit with the numpy restatement the oracle loop uses,
and two oracle steps keep the loop's invariants (mass, plate contact)."""
import numpy as np
import pytest

from paper_2405_13165_gb300 import clouds as C

torch = pytest.importorskip("torch")

import tray_oracle as TO  # noqa: E402
from paper_2405_13165_gb300 import tray  # noqa: E402


def _cloud():
    return C.tray_cloud(0.02)


def test_displacement_and_advection_bitwise_equal():
    c = _cloud()
    vel = C.tray_velocity(c.dx)
    P = c.pos_h.copy()
    d_np = TO.displacement(P[:, :3], vel)
    d_t = tray.displacement(torch.from_numpy(P[:, :3].copy()), vel).numpy()
    assert d_np.dtype == np.float32
    np.testing.assert_array_equal(d_np, d_t)
    assert np.abs(d_np).max() <= 0.2 * c.dx * (1 + 1e-6)
    s = TO.initial_state(c)
    TO.advect(s, vel)
    pt = torch.from_numpy(c.pos_h.copy())
    tray.advect(pt, torch.from_numpy(c.model), torch.from_numpy(c.ptype), vel)
    np.testing.assert_array_equal(s["pos_h"], pt.numpy())
    planar = (c.model == C.MODEL_2D) | (c.ptype == C.TYPE_WALL)
    assert np.all(s["pos_h"][planar, 2] == c.pos_h[planar, 2])


@pytest.mark.parametrize("k", [0, 7, 19])
def test_user_criterion_equal(k):
    c = _cloud()
    u_np = TO.user_flags(c.pos_h, c.model, k)
    u_t = tray.user_flags(torch.from_numpy(c.pos_h), torch.from_numpy(c.model), k).numpy()
    np.testing.assert_array_equal(u_np, u_t)
    assert np.all(u_np[c.model == C.MODEL_3D] != C.USER_TO_3D)
    assert np.all(u_np[c.model == C.MODEL_2D] != C.USER_TO_2D)


def test_oracle_loop_conserves_mass_and_keeps_plate_contact(orc):
    c = C.tray_cloud(0.03)
    vel = C.tray_velocity(c.dx)
    s = TO.initial_state(c)
    m0 = s["mass"].astype(np.float64).sum()
    switched = 0
    for k in range(2):
        s, info = TO.step(s, k, vel)
        switched += int((info["flag"] != 0).sum())
        planar = (s["model"] == C.MODEL_2D) | (s["ptype"] == C.TYPE_WALL)
        assert np.all(s["pos_h"][planar, 2] == 0.0)
        assert np.all(s["pos_h"][~planar, 2] >= vel["zmin"])
    assert switched > 0
    assert abs(s["mass"].astype(np.float64).sum() - m0) <= 1e-5 * m0
