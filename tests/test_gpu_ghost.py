"""The buffer zone (Sec. 5.3, Alg. 5) on the GPU through the C ABI, stage by
stage against the oracle: sources, intermediate ghosts, the ghost cloud's
neighbours and transition, the union, and the regular particles' stencils and
derivatives over regular plus ghost neighbours."""
import numpy as np
import pytest

from paper_2405_13165_gb300 import clouds as C

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2405_13165_gb300 import mafp as M  # noqa: E402
from paper_2405_13165_gb300.ghosts import GhostZone, empty_state  # noqa: E402
from paper_2405_13165_gb300.pipeline import Pipeline  # noqa: E402
from parity_util import (TOL, outputs_vs_bar, sensitivity,  # noqa: E402
                         stencil_rowwise_error_vec)

KEYMAP = {"type": "ptype"}


def _state(c, cap, dtype):
    s = empty_state(cap, dtype)
    rd = M.real_dtype(dtype)
    for k, v in s.items():
        a = np.asarray(getattr(c, KEYMAP.get(k, k)))
        v[: c.n] = torch.from_numpy(a).to(v.device, rd if v.is_floating_point() else torch.uint8)
    return s


@pytest.mark.parametrize("dtype", [M.F32_REFINED, M.F64])
@pytest.mark.parametrize("dx,columns", [(0.02, True), (0.008, False)])
def test_ghost_zone_matches_oracle(orc, dtype, dx, columns):
    c = C.interface_strip(dx=dx, quadratic=columns, columns=columns)
    n = c.n
    cap = 2 * n
    ctx = M.Context(cap)
    S = _state(c, cap, dtype)
    pipe = Pipeline(ctx, cap, 400 * cap, dtype)
    d = {"pos_h": S["pos_h"][:n]}
    pipe.neighbours(d)
    rp, col = pipe.csr(n)
    gz = GhostZone(ctx, cap, n, 4 * n, 400 * n, dtype)
    n_all, ng, ngo = gz.build(S, n, rp, col)
    # oracle
    o_rp, o_col = orc.neighbours(c.pos_h)
    np.testing.assert_array_equal(rp.cpu().numpy(), o_rp)
    ost = orc.cloud_state(c)
    if dtype == M.F64:     # the FP64 path keeps the ghosts' data in FP64
        ost = {k: (np.asarray(v, np.float64) if np.asarray(v).dtype == np.float32 else v)
               for k, v in ost.items()}
    u, src, gflag, o_ng = orc.ghost_zone(ost, o_rp, o_col)
    np.testing.assert_array_equal(gz.src[:n].cpu().numpy(), src)
    assert ng == o_ng
    np.testing.assert_array_equal(gz.flag[:ng].cpu().numpy(), gflag)
    np.testing.assert_array_equal(gz.ghost_src[:ng].cpu().numpy(), np.nonzero(src)[0])
    assert n_all == len(u["model"])
    for k in ("model", "last"):
        np.testing.assert_array_equal(S[k][:n_all].cpu().numpy(), u[k])
    np.testing.assert_array_equal(S["type"][:n_all].cpu().numpy(), u["ptype"])
    tol = 1e-6 if dtype != M.F64 else 1e-13
    for k in ("pos_h", "vp", "mass", "hfilm", "rho"):
        a = S[k][:n_all].double().cpu().numpy()
        b = np.asarray(u[k], np.float64)
        assert np.all(np.abs(a - b).max(0) <= tol * np.maximum(np.abs(b).max(0), 1e-30)), k
    # derivatives at the regular particles over regular + ghost neighbours
    U = {k: S[k][:n_all] for k in S}
    du = {"pos_h": U["pos_h"], "model": U["model"], "ptype": U["type"], "normal": U["normal"],
          "vol": (U["mass"] / U["rho"]).contiguous(), "h3d": U["h3d"],
          "user": torch.zeros(n_all, dtype=torch.uint8, device="cuda"), "last": U["last"],
          "fields": U["vp"]}
    pipe.neighbours(du)
    pipe.classify(du)            # film frames
    pipe.stencils(du)
    pipe.apply(du)
    torch.cuda.synchronize()
    assert ctx.status()["code"] == 0
    g_rp, g_col = pipe.csr(n_all)
    P = np.asarray(u["pos_h"], np.float64)
    ur, ucol = orc.neighbours(P)
    np.testing.assert_array_equal(g_rp.cpu().numpy(), ur)
    np.testing.assert_array_equal(g_col.cpu().numpy(), ucol)
    rows = np.arange(n)
    coef, status, _ = orc.stencils(P, u["model"], ur, ucol, rows=rows)
    out = orc.apply(ur, ucol, coef, u["vp"], rows=rows)
    e_reg = int(ur[n])
    gcoef = pipe.coef[:e_reg].double().cpu().numpy()
    err, _ = stencil_rowwise_error_vec(ur[: n + 1], gcoef, coef[:e_reg])
    assert np.all(err <= TOL[dtype]), err
    # the depth-constant quadratic fields have d/dz = 0 (columns that are zero
    # to rounding) and a constant Laplacian that is a small difference of large
    # terms: the outputs that miss the plain bar are counted and each bounded
    # by the roundoff of its terms
    gout = pipe.out[:n].double().cpu().numpy()
    sens = sensitivity(ur, ucol, coef, u["vp"], rows=rows)[:n]
    # FP64: the union's ghosts went through the remap in both paths and agree
    # to `tol` (checked above), not to the last bit
    r = outputs_vs_bar(gout, out[:n], sens, dtype, unit=tol if dtype == M.F64 else None)
    print(f"outputs above the plain bar {r['above']} of {r['outputs']}, worst exception "
          f"{r['worst_exception']:.3g} of its bound, zero columns {r['zero_columns']}")
    assert r["ok"], r
    ctx.close()


def test_ghost_capacity_reported():
    c = C.interface_strip(dx=0.02)
    n = c.n
    ctx = M.Context(2 * n)
    S = _state(c, 2 * n, M.F32_REFINED)
    pipe = Pipeline(ctx, 2 * n, 400 * n, M.F32_REFINED)
    pipe.neighbours({"pos_h": S["pos_h"][:n]})
    rp, col = pipe.csr(n)
    gz = GhostZone(ctx, 2 * n, 8, 64, 4096)            # far too few ghost rows
    with pytest.raises(M.MafpError):
        gz.build(S, n, rp, col)
    torch.cuda.synchronize()
    assert ctx.status()["code"] == M.ECAPACITY
    ctx.close()
