"""Pins of the advection-diffusion workload's CPU side: the analytic reference
and the oracle loop's exact transport (Sec. 7.2: with kappa = 0 the data
transfer between the models must reproduce the transported disc exactly)."""
import numpy as np
import pytest

from paper_2405_13165_gb300 import clouds as C

import advdiff_oracle as AO  # noqa: E402


def test_exact_temperature_closed_forms():
    x0, y0, R = C.ADV_DISC
    # heat is conserved: the plane integral of T stays the disc area
    g = np.linspace(0.25, 1.75, 151)
    X, Y = np.meshgrid(g, np.linspace(-0.25, 1.25, 151), indexing="ij")
    xy = np.stack([X.ravel(), Y.ravel()], 1)
    T = AO.exact_temperature(xy, 0.5, 5e-3, nr=32, nt=64)
    cell = (g[1] - g[0]) ** 2
    assert abs(T.sum() * cell - np.pi * R * R) <= 1e-3 * np.pi * R * R
    # centre value: 1 - exp(-R^2 / (4 kappa t)) (radial integral of the kernel)
    for t, k in ((0.5, 5e-3), (2.0, 5e-3), (1.0, 0.02)):
        c = AO.exact_temperature(np.array([[x0 + t, y0]]), t, k)[0]
        assert abs(c - (1.0 - np.exp(-R * R / (4 * k * t)))) <= 1e-10
    # kappa = 0: the moved indicator
    pts = np.array([[x0 + 1.0, y0], [x0 + 1.0 + 0.21, y0]])
    np.testing.assert_array_equal(AO.exact_temperature(pts, 1.0, 0.0), [1.0, 0.0])


def test_oracle_pure_advection_is_exact(orc):
    c = C.advection_plate(0.4)
    s = AO.initial_state(c)
    seen3d = False
    for _ in range(200):
        s, info = AO.step(s, 0.01, 0.0)
        seen3d |= bool((s["model"] == C.MODEL_3D).any())
    assert seen3d
    T = s["vp"][:, 0].astype(np.float64)
    Tref = AO.exact_temperature(s["pos_h"][:, :2].astype(np.float64), 2.0, 0.0)
    np.testing.assert_array_equal(T, Tref)
