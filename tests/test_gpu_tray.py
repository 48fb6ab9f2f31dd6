"""The tray loop on the GPU (config 5 workload): a short trajectory against the
oracle's own trajectory (the oracle runs every stage and the workload rules in
numpy float32 itself), and the full 16M-particle, 20-step loop checked at step
0 against the oracle and on invariants at every step."""
import numpy as np
import pytest

from paper_2405_13165_gb300 import clouds as C

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import oracle as O  # noqa: E402
import tray_oracle as TO  # noqa: E402
from paper_2405_13165_gb300 import mafp as M, tray  # noqa: E402
from parity_util import outputs_vs_bar, sensitivity  # noqa: E402


def _pairs(rp, col):
    rows = np.repeat(np.arange(len(rp) - 1, dtype=np.int64), np.diff(rp))
    return rows * (len(rp) - 1) + col.astype(np.int64)


def _csr_agree(g_rp, g_col, o_rp, o_col, P):
    """Equal, except pairs within 1e-5 (relative) of the support boundary
    (the trajectories may differ in the last bit of a remapped position)."""
    n = len(o_rp) - 1
    diff = np.setxor1d(_pairs(g_rp, g_col), _pairs(o_rp, o_col), assume_unique=True)
    i, j = diff // n, diff % n
    Pd = P.astype(np.float64)
    d2 = ((Pd[j, :3] - Pd[i, :3]) ** 2).sum(1)
    r2 = (0.5 * (Pd[i, 3] + Pd[j, 3])) ** 2
    assert np.all(np.abs(d2 - r2) <= 1e-5 * r2), diff[:10]
    return diff.size


def test_tray_trajectory_matches_oracle_trajectory(orc):
    c = C.config_tray(300_000)
    vel = C.tray_velocity(c.dx)
    n0 = c.n
    ctx = M.Context(2 * n0)
    loop = tray.TrayLoop(ctx, c, cap=2 * n0, cap_nnz=400 * n0)
    s = TO.initial_state(c)
    switched = 0
    for k in range(3):
        n = loop.n
        assert n == len(s["model"])
        st = loop.step(k)
        nxt, info = TO.step(s, k, vel)
        p = loop.pipe
        g_rp = p.row_ptr[: n + 1].cpu().numpy()
        g_col = p.col[: int(g_rp[-1])].cpu().numpy()
        ndiff = _csr_agree(g_rp, g_col, info["row_ptr"], info["col"], s["pos_h"])
        if k == 0:
            assert ndiff == 0
        far = info["near"] == 0
        np.testing.assert_array_equal(p.flag[:n].cpu().numpy()[far], info["flag"][far])
        assert np.all(info["near"] == 0)                # otherwise the trajectories part
        # thin 3D layers give near-degenerate rows with large cancelling
        # coefficients: the few outputs that miss the plain bar are counted
        # and each bounded by the roundoff of its terms
        sens = sensitivity(info["row_ptr"], info["col"], info["coef"], s["vp"])
        r = outputs_vs_bar(p.out[:n].double().cpu().numpy(), info["out"], sens, M.F32_REFINED)
        print(f"step {k}: outputs above the plain bar {r['above']} of {r['outputs']}, "
              f"worst exception {r['worst_exception']:.3g} of its bound, "
              f"componentwise p99 max {r['p99'].max():.3g}")
        assert r["ok"], (k, r)
        assert st["n_out"] == info["n_out"]
        np.testing.assert_array_equal(loop.old2new[:n].cpu().numpy(), info["old2new"])
        G = loop.cur
        m = st["n_out"]
        for key in ("model", "last"):
            np.testing.assert_array_equal(G[key][:m].cpu().numpy(), nxt[key])
        np.testing.assert_array_equal(G["type"][:m].cpu().numpy(), nxt["ptype"])
        for key in ("pos_h", "vp", "mass", "rho", "hfilm"):
            a = G[key][:m].double().cpu().numpy()
            b = nxt[key].astype(np.float64)
            scale = np.abs(b).max(0)
            assert np.all(np.abs(a - b).max(0) <= 1e-6 * np.maximum(scale, 1e-30)), key
        switched += st["to2d"] + st["to3d"]
        s = nxt
    assert switched > 0
    assert ctx.status()["code"] == 0
    ctx.close()


def test_tray_full_size_twenty_steps(orc):
    c = C.config_tray()                                  # 16M particles
    n0 = c.n
    rp, col = O.neighbours(c.pos_h)
    cap = int(1.35 * n0)
    ctx = M.Context(cap)
    loop = tray.TrayLoop(ctx, c, cap=cap, cap_nnz=int(1.35 * rp[-1]))
    m0 = loop.mass()
    # step 0 from the generator's cloud: neighbours and flags in full, stencils
    # and outputs on a seeded 1 % of the rows, against the oracle
    vel = C.tray_velocity(c.dx)
    user = TO.user_flags(c.pos_h, c.model, 0)
    st = loop.step(0)
    p = loop.pipe
    np.testing.assert_array_equal(p.row_ptr[: n0 + 1].cpu().numpy(), rp)
    np.testing.assert_array_equal(p.col[: rp[-1]].cpu().numpy(), col)
    cl = O.classify(c.pos_h, c.model, c.ptype, c.normal, c.vol, c.h3d, user, rp, col)
    flag = O.smooth(c.model, cl["preflag"], c.last, rp, col)
    far = cl["near"] == 0
    np.testing.assert_array_equal(p.flag[:n0].cpu().numpy()[far], flag[far])
    rows = np.sort(np.random.default_rng(55).choice(n0, n0 // 100, replace=False))
    coef, status, _ = O.stencils(c.pos_h, c.model, rp, col, rows=rows)
    out = O.apply(rp, col, coef, c.vp, rows=rows)
    sens = sensitivity(rp, col, coef, c.vp, rows=rows)
    r = outputs_vs_bar(p.out[:n0].double().cpu().numpy()[rows], out[rows], sens[rows],
                       M.F32_REFINED)
    print(f"16M step 0: outputs above the plain bar {r['above']} of {r['outputs']}, "
          f"worst exception {r['worst_exception']:.3g} of its bound, "
          f"componentwise p99 max {r['p99'].max():.3g}")
    assert r["ok"], r
    # twenty steps: invariants at every step
    stats = [st]
    for k in range(1, 20):
        stats.append(loop.step(k))
        assert ctx.status()["code"] == 0
    for s in stats:
        assert s["n_out"] == s["n_in"] - s["deleted"] + s["added"]
    frac = [(s["to2d"] + s["to3d"] + s["deleted"] + s["added"]) / s["n_in"] for s in stats]
    print("switching fraction per step:", np.round(frac, 4).tolist())
    assert 0.01 <= float(np.mean(frac)) <= 0.15
    assert abs(loop.mass() - m0) <= 1e-4 * m0
    n = loop.n
    P = loop.cur["pos_h"][:n]
    planar = (loop.cur["model"][:n] == M.MODEL_2D) | (loop.cur["type"][:n] == M.TYPE_WALL)
    assert bool((P[planar, 2] == 0).all())
    ctx.close()
