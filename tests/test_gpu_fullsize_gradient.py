"""Differentiation at full size: the 2M-particle cube-on-sheet cloud (dx bisected
to 2M).  Loss L = sum over all rows of the squared Laplacians of the four
fields.  The GPU gradients with respect to the particle positions (stencil
adjoint, film frames included) and the field values (apply transpose) are
compared with the FP64 oracle on every particle, and the FP64 GPU gradient with
central finite differences of the FP64 GPU forward (step 1e-4 dx, neighbour
sets held fixed, film frames recomputed from the moved positions) on every
coordinate."""
import numpy as np
import pytest

from paper_2405_13165_gb300 import clouds as C

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import oracle as O  # noqa: E402
from paper_2405_13165_gb300 import mafp as M  # noqa: E402
from paper_2405_13165_gb300.pipeline import Pipeline, cloud_to_device  # noqa: E402
from parity_util import TOL  # noqa: E402

@pytest.fixture(scope="module")
def diff2m():
    c = C.cell_sorted(C.config_diff_2m())
    rp, col = O.neighbours(c.pos_h)
    coef, status, _ = O.stencils(c.pos_h, c.model, rp, col)
    out = O.apply(rp, col, coef, c.vp)
    G = np.zeros_like(out)
    G[:, :, 3] = 2.0 * out[:, :, 3]          # dL/dout of L = sum_i sum_f (Lap_i f)^2
    gpos = O.stencil_grad(c.pos_h, c.model, rp, col, c.vp, G)
    gfld = O.apply_T(rp, col, coef, G)
    return c, rp, col, G, gpos, gfld


def _gpu(c, dtype, cap):
    ctx = M.Context(c.n)
    pipe = Pipeline(ctx, c.n, cap, dtype)
    d = cloud_to_device(c, dtype)
    ctx.reset_status()
    pipe.step(d)
    torch.cuda.synchronize()
    return ctx, pipe, d


@pytest.mark.parametrize("dtype", [M.F32_REFINED, M.F64])
def test_gradients_match_oracle_on_every_particle(diff2m, dtype):
    c, rp, col, G, o_gpos, o_gfld = diff2m
    n = c.n
    ctx, pipe, d = _gpu(c, dtype, int(rp[-1]) + 1024)
    assert ctx.status()["code"] == 0
    g_rp, g_col = pipe.csr(n)
    np.testing.assert_array_equal(g_rp.cpu().numpy(), rp)
    np.testing.assert_array_equal(g_col.cpu().numpy(), col)
    rd = M.real_dtype(dtype)
    gout = torch.tensor(G, dtype=rd, device="cuda")
    gpos = torch.empty(n, 4, dtype=rd, device="cuda")
    gfld = torch.empty(n, 4, dtype=rd, device="cuda")
    M.build_stencils_backward(ctx, d["pos_h"], d["model"], pipe.frame[:n], g_rp, g_col,
                              d["fields"], gout, gpos, dtype)
    M.apply_ops_backward(ctx, g_rp, g_col, None, pipe.coef, gout, gfld, dtype)
    torch.cuda.synchronize()
    assert ctx.status()["code"] == 0
    a = gpos.double().cpu().numpy()
    tol = 2e-3 if dtype != M.F64 else 1e-8
    scale = np.abs(o_gpos[:, :3]).max(0)
    err = np.abs(a[:, :3] - o_gpos[:, :3]).max(0) / scale
    assert np.all(err <= tol), err
    assert np.all(a[:, 3] == 0)
    f = gfld.double().cpu().numpy()
    fscale = np.abs(o_gfld).max(0)
    ferr = np.abs(f - o_gfld).max(0) / fscale
    assert np.all(ferr <= TOL[dtype]), ferr
    ctx.close()


def test_fp64_gradient_matches_central_differences(diff2m):
    c, rp, col, *_ = diff2m
    n = c.n
    ctx, pipe, d = _gpu(c, M.F64, int(rp[-1]) + 1024)
    g_rp, g_col = pipe.csr(n)
    G = torch.zeros(n, 4, 4, dtype=torch.float64, device="cuda")
    G[:, :, 3] = 2.0 * pipe.out[:n, :, 3]
    gpos = torch.empty(n, 4, dtype=torch.float64, device="cuda")
    pos = d["pos_h"].clone()
    M.build_stencils_backward(ctx, pos, d["model"], pipe.frame[:n], g_rp, g_col, d["fields"], G,
                              gpos, M.F64)
    g = gpos.cpu().numpy()

    def local_loss(p, rows_t):
        # moving particle k changes only the rows that hold k (and their film
        # frames), so the change of L is the change of its sum over those rows
        pipe.classify(dict(d, pos_h=p))
        pipe.stencils(dict(d, pos_h=p))
        pipe.apply(dict(d, pos_h=p))
        return float((pipe.out[rows_t, :, 3] ** 2).sum().item())

    P = c.pos_h.astype(np.float64)
    step = 1e-4 * c.dx
    rng = np.random.default_rng(45)
    film = np.nonzero(c.model == 1)[0]
    bulk = np.nonzero(c.model == 0)[0]
    cand = np.concatenate([rng.choice(film, 200, replace=False), rng.choice(bulk, 200, replace=False)])
    checked = film_z = 0
    for k in cand:
        r = col[rp[k]:rp[k + 1]]
        dist = np.linalg.norm(P[r, :3] - P[k, :3], axis=1)
        if np.any(np.abs(dist - 0.5 * (P[r, 3] + P[k, 3])) <= 10 * step):
            continue
        rows_t = torch.tensor(r.astype(np.int64), device="cuda")
        for a in (0, 1, 2):
            pp, pm = pos.clone(), pos.clone()
            pp[k, a] += step
            pm[k, a] -= step
            fd = (local_loss(pp, rows_t) - local_loss(pm, rows_t)) / (2 * step)
            scale = max(abs(fd), 1e-3 * np.abs(g[:, :3]).max())
            assert abs(g[k, a] - fd) <= 1e-4 * scale + 1e-9, (k, a, g[k, a], fd)
            checked += 1
            film_z += int(c.model[k] == 1 and a == 2)
        if checked >= 48 and film_z >= 12:
            break
    assert checked >= 48 and film_z >= 12
    ctx.close()
