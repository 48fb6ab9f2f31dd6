"""Parity at the benchmark's full size: the 1M-particle jet-on-plate cloud in
cell order, with the launch shapes the autotuner picks (the configuration the
benchmark times).  Neighbour lists and flags are compared in full; stencils
and applied derivatives on a seeded sample of rows the oracle computes one by
one; properties that hold at any size are checked on everything."""
import numpy as np
import pytest

from paper_2405_13165_gb300 import clouds as C

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import oracle as O  # noqa: E402
from paper_2405_13165_gb300 import autotune, mafp as M  # noqa: E402
from paper_2405_13165_gb300.pipeline import Pipeline, cloud_to_device  # noqa: E402
from parity_util import P99_BAR, TOL, column_error  # noqa: E402


@pytest.fixture(scope="module")
def jet():
    c = C.cell_sorted(C.config_jet_1m())
    rp, col = O.neighbours(c.pos_h)
    return c, rp, col


@pytest.fixture(scope="module")
def gpu_run(jet):
    c, orp, ocol = jet
    n = c.n
    ctx = M.Context(n)
    pipe = Pipeline(ctx, n, int(orp[-1]) + 1024, M.F32_REFINED)
    d = cloud_to_device(c)
    tuned = autotune.tune(ctx, pipe, d, use_cache=False)
    ctx.reset_status()
    pipe.step(d)
    torch.cuda.synchronize()
    st = ctx.status()
    nnz = int(pipe.row_ptr[n].item())
    res = dict(row_ptr=pipe.row_ptr[: n + 1].cpu().numpy(), col=pipe.col[:nnz].cpu().numpy(),
               flag=pipe.flag[:n].cpu().numpy(), preflag=pipe.preflag[:n].cpu().numpy(),
               coef=pipe.coef[:nnz], out=pipe.out[:n].double().cpu().numpy(),
               status=pipe.status[:n].cpu().numpy(), st=st, tuning=tuned)
    return res


def test_neighbours_bit_exact_full(jet, gpu_run):
    c, orp, ocol = jet
    assert gpu_run["st"]["code"] == 0 and gpu_run["st"]["cells_identity"] == 1
    np.testing.assert_array_equal(gpu_run["row_ptr"], orp)
    np.testing.assert_array_equal(gpu_run["col"], ocol)


def test_flags_bit_exact_full(jet, gpu_run):
    c, rp, col = jet
    cl = O.classify(c.pos_h, c.model, c.ptype, c.normal, c.vol, c.h3d, c.user, rp, col)
    flag = O.smooth(c.model, cl["preflag"], c.last, rp, col)
    far = cl["near"] == 0
    np.testing.assert_array_equal(gpu_run["preflag"][far], cl["preflag"][far])
    np.testing.assert_array_equal(gpu_run["flag"][far], flag[far])


def test_stencils_and_outputs_on_sampled_rows(jet, gpu_run):
    c, rp, col = jet
    rng = np.random.default_rng(2405)
    rows = np.sort(rng.choice(c.n, 3000, replace=False))
    coef, status, _ = O.stencils(c.pos_h, c.model, rp, col, rows=rows)
    out = O.apply(rp, col, coef, c.vp, rows=rows)
    gcoef = gpu_run["coef"]
    worst = np.zeros(4)
    for i in rows:
        s, e = rp[i], rp[i + 1]
        a = gcoef[s:e].double().cpu().numpy()
        b = coef[s:e]
        scale = np.abs(b).max(0)
        ok = scale > 0
        worst[ok] = np.maximum(worst[ok], np.abs(a - b).max(0)[ok] / scale[ok])
    assert np.all(worst <= TOL[M.F32_REFINED]), worst
    np.testing.assert_array_equal(gpu_run["status"][rows] == M.STENCIL_DEFICIENT, status[rows] == 1)
    a = gpu_run["out"][rows].reshape(-1, 16)
    b = out[rows].reshape(-1, 16)
    nw = np.abs(a - b).max(0) / np.abs(b).max(0)
    assert np.all(nw <= TOL[M.F32_REFINED]), nw
    # componentwise p99 (floor 1e-3 of the column maximum)
    _, p99 = column_error(a, b)
    print("componentwise p99 per column:", np.array2string(p99, precision=2))
    assert np.all(p99 <= P99_BAR[M.F32_REFINED]), p99


def test_stencil_properties_on_all_rows(jet, gpu_run):
    # properties at any size: every row of a non-deficient stencil annihilates
    # constants and differentiates the linear monomials exactly (to FP32)
    c, rp, col = jet
    n = c.n
    rp_t = torch.tensor(rp, device="cuda")
    rows = torch.repeat_interleave(torch.arange(n, device="cuda"), rp_t[1:] - rp_t[:-1])
    colt = torch.tensor(col.astype(np.int64), device="cuda")
    coef = gpu_run["coef"].double()
    X = torch.tensor(c.pos_h[:, :3].astype(np.float64), device="cuda")
    h = torch.tensor(c.pos_h[:, 3].astype(np.float64), device="cuda")
    ok = torch.tensor(gpu_run["status"] != M.STENCIL_DEFICIENT, device="cuda")
    s0 = torch.zeros(n, 4, dtype=torch.float64, device="cuda").index_add_(0, rows, coef)
    scale0 = torch.zeros(n, 4, dtype=torch.float64, device="cuda").index_add_(0, rows, coef.abs())
    assert torch.all((s0.abs() <= 1e-5 * scale0)[ok])
    d = X[colt] - X[rows]
    for a in range(3):
        g = torch.zeros(n, dtype=torch.float64, device="cuda").index_add_(0, rows, coef[:, a] * d[:, a])
        model = torch.tensor(c.model, device="cuda")
        m3 = ok & (model == 0)
        assert torch.all((g[m3] - 1.0).abs() <= 1e-4), float((g[m3] - 1.0).abs().max())


def test_outputs_on_all_rows(jet, gpu_run):
    # every applied derivative of the cloud against the FP64 oracle (stencils
    # and apply over all rows): the 1e-4 normwise bar and the componentwise
    # p99 bar on each of the 16 columns (field x operator)
    c, rp, col = jet
    coef, status, _ = O.stencils(c.pos_h, c.model, rp, col)
    out = O.apply(rp, col, coef, c.vp).reshape(-1, 16)
    a = gpu_run["out"].reshape(-1, 16)
    nw, p99 = column_error(a, out)
    print("normwise per column:", np.array2string(nw, precision=2))
    print("componentwise p99 per column:", np.array2string(p99, precision=2))
    assert np.all(nw <= TOL[M.F32_REFINED]), nw
    assert np.all(p99 <= P99_BAR[M.F32_REFINED]), p99
