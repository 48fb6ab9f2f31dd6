"""Advection-diffusion over the plate with a 3D band (Eq. AdvDiff, Sec. 7.2)
on the GPU: the whole 200-step trajectory against the oracle's own trajectory,
exact transport without diffusion, and convergence towards the analytic
solution under refinement."""
import numpy as np
import pytest

from paper_2405_13165_gb300 import clouds as C

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import advdiff_oracle as AO  # noqa: E402
from paper_2405_13165_gb300 import advdiff as A, mafp as M  # noqa: E402


def _loop(c, kappa, dt):
    cap = 3 * c.n
    ctx = M.Context(cap)
    return ctx, A.AdvDiffLoop(ctx, c, kappa, dt, cap, 300 * cap)


def test_trajectory_matches_oracle(orc):
    h, kappa = 0.2, 5e-3
    c = C.advection_plate(h)
    dt = A.time_step(h, kappa)
    ctx, loop = _loop(c, kappa, dt)
    s = AO.initial_state(c)
    for k in range(int(round(2.0 / dt))):
        st = loop.step()
        s, info = AO.step(s, dt, kappa)
        assert np.all(info["near"] == 0)
        assert st["n"] == info["n"] and st["n_all"] == info["n_all"], (k, st, info)
        if k % 20 == 0 or k == 199:
            n = loop.n
            G = loop.cur
            np.testing.assert_array_equal(G["model"][:n].cpu().numpy(), s["model"])
            np.testing.assert_array_equal(G["pos_h"][:n].cpu().numpy(), s["pos_h"])
            T = G["vp"][:n, 0].double().cpu().numpy()
            assert np.abs(T - s["vp"][:, 0]).max() <= 1e-4, k
    assert ctx.status()["code"] == 0
    ctx.close()


def test_pure_advection_exact():
    c = C.advection_plate(0.1)
    ctx, loop = _loop(c, 0.0, 0.01)
    three_d = 0
    for _ in range(200):
        st = loop.step()
        three_d = max(three_d, st["n_all"] - st["ghosts"])
    P, T, model = loop.temperature()
    np.testing.assert_array_equal(T, AO.exact_temperature(P[:, :2], 2.0, 0.0))
    ctx.close()


def test_convergence_to_analytic_solution():
    kappa = 5e-3
    res = []
    for h in (0.4, 0.2, 0.1, 0.05):
        c = C.advection_plate(h)
        dt = A.time_step(h, kappa)
        ctx, loop = _loop(c, kappa, dt)
        for _ in range(int(round(2.0 / dt))):
            loop.step()
        assert ctx.status()["code"] == 0
        P, T, model = loop.temperature()
        e2, einf = AO.errors(T, AO.exact_temperature(P[:, :2], 2.0, kappa))
        res.append((h, c.n, e2, einf))
        ctx.close()
    print("h, N, eps2, epsinf:", res)
    e2 = [r[2] for r in res]
    assert all(b < a for a, b in zip(e2, e2[1:])), res
    assert e2[-1] < 0.25 * e2[1], res
