"""Film momentum step and post-processing kernels through the C ABI against
the oracle's formulas, on the jet-on-plate cloud's own stencil outputs."""
import numpy as np
import pytest

from paper_2405_13165_gb300 import clouds as C

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2405_13165_gb300 import mafp as M  # noqa: E402
from parity_util import run_gpu  # noqa: E402


@pytest.mark.parametrize("dtype", [M.F32_REFINED, M.F64])
def test_film_momentum_and_post_processing(orc, dtype):
    c = C.config_small()
    g, pipe, d, ctx = run_gpu(c, dtype)
    n = c.n
    rd = M.real_dtype(dtype)
    out = pipe.out[:n].contiguous()
    out_h = out.double().cpu().numpy()
    hfilm = pipe.hfilm[:n].contiguous()
    tol = 1e-6 if dtype != M.F64 else 1e-13
    # film momentum with the film heights the detection computed
    vp = d["vp"].clone()
    M.film_momentum(ctx, d["model"], vp, d["rho"], d["eta"], hfilm, d["normal"], out,
                    [0.0, 0.5, -9.81], 1e-3, dtype)
    want = orc.film_momentum(c.model, c.vp, c.rho, c.eta, hfilm.double().cpu().numpy(),
                             c.normal, out_h, [0.0, 0.5, -9.81], 1e-3)
    got = vp.double().cpu().numpy()
    assert np.all(np.abs(got - want).max(0) <= tol * np.maximum(np.abs(want).max(0), 1e-30))
    # plane flux over a displacement
    p0 = d["pos_h"]
    p1 = p0.clone()
    p1[:, 0] += 0.013
    acc = torch.zeros(2, dtype=torch.float64, device="cuda")
    M.plane_flux(ctx, p0, p1, d["mass"], d["rho"], [0.5, 0.0, 0.0], [1.0, 0.0, 0.0], acc, dtype)
    vol, cnt = orc.plane_flux(p0.double().cpu().numpy(), p1.double().cpu().numpy(), c.mass,
                              c.rho, [0.5, 0, 0], [1, 0, 0])
    a = acc.cpu().numpy()
    assert int(a[1]) == cnt > 0
    assert abs(a[0] - vol) <= 1e-9 * abs(vol)
    # n^T S n over the plate's 3D wall particles
    sel = torch.tensor(((c.model == 0) & (c.ptype == 2)).astype(np.uint8), device="cuda")
    acc.zero_()
    M.normal_stress(ctx, sel, out, d["eta"], d["normal"], acc, dtype)
    s, cnt = orc.normal_stress(sel.cpu().numpy(), out_h, c.eta, c.normal)
    a = acc.cpu().numpy()
    assert int(a[1]) == cnt > 0
    assert abs(a[0] - s) <= 1e-6 * max(abs(s), 1e-30)
    ctx.close()
