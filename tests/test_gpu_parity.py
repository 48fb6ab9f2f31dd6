"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on the
same seeded inputs.  Neighbour sets and flags bit-exact (flags within 1e-6 of a
threshold counted, not compared); stencils / outputs within the tolerances of
parity_util.TOL."""
import numpy as np
import pytest

from paper_2405_13165_gb300 import clouds as C

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2405_13165_gb300 import mafp as M  # noqa: E402
from parity_util import (P99_BAR, TOL, column_error, run_gpu,  # noqa: E402
                         stencil_rowwise_error_vec)

DTYPES = [M.F32_REFINED, M.F64]


def _oracle_all(orc, c):
    rp, col = orc.neighbours(c.pos_h)
    cl = orc.classify(c.pos_h, c.model, c.ptype, c.normal, c.vol, c.h3d, c.user, rp, col)
    flag = orc.smooth(c.model, cl["preflag"], c.last, rp, col)
    coef, status, cond = orc.stencils(c.pos_h, c.model, rp, col)
    out = orc.apply(rp, col, coef, c.vp)
    return dict(row_ptr=rp, col=col, flag=flag, coef=coef, status=status, cond=cond, out=out, **cl)


def _check_csr(g, o):
    np.testing.assert_array_equal(g["row_ptr"], o["row_ptr"])
    np.testing.assert_array_equal(g["col"], o["col"])


def _check_flags(g, o):
    far = o["near"] == 0
    np.testing.assert_array_equal(g["preflag"][far], o["preflag"][far])
    np.testing.assert_array_equal(g["flag"][far], o["flag"][far])


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("sort", [False, True])
def test_small_config_end_to_end(orc, dtype, sort):
    c = C.config_small()
    if sort:
        c = C.cell_sorted(c)
    o = _oracle_all(orc, c)
    g, *_ = run_gpu(c, dtype)
    assert g["status_block"]["code"] == 0
    assert g["status_block"]["cells_identity"] == int(sort)
    _check_csr(g, o)
    _check_flags(g, o)
    np.testing.assert_array_equal(g["status"] != M.STENCIL_DEFICIENT, o["status"] == 0)
    err, _ = stencil_rowwise_error_vec(o["row_ptr"], g["coef"], o["coef"])
    assert np.all(err <= TOL[dtype]), err
    nw, p99 = column_error(g["out"], o["out"])
    assert np.all(nw <= TOL[dtype]), (nw, p99)
    assert np.all(p99 <= P99_BAR[dtype]), p99


def test_plain_fp32_is_worse_than_refined(orc):
    c = C.config_small()
    o = _oracle_all(orc, c)
    gr, *_ = run_gpu(c, M.F32_REFINED)
    gp, *_ = run_gpu(c, M.F32_PLAIN)
    er, _ = stencil_rowwise_error_vec(o["row_ptr"], gr["coef"], o["coef"])
    ep, _ = stencil_rowwise_error_vec(o["row_ptr"], gp["coef"], o["coef"])
    assert er.max() < ep.max()
    assert ep.max() <= TOL[M.F32_PLAIN]


@pytest.mark.parametrize("seed", [0, 1])
@pytest.mark.parametrize("dtype", DTYPES)
def test_random_cloud_variable_h_unsorted(orc, seed, dtype):
    # random order (row sort path), variable support radii, mixed models/types
    c = C.random_cloud(6000, seed=seed, h_lo=0.05, h_hi=0.11)
    rp, col = orc.neighbours(c.pos_h)
    g, *_ = run_gpu(c, dtype, stages=("nbr", "cls"))
    _check_csr(g, dict(row_ptr=rp, col=col))
    cl = orc.classify(c.pos_h, c.model, c.ptype, c.normal, c.vol, c.h3d, c.user, rp, col)
    flag = orc.smooth(c.model, cl["preflag"], c.last, rp, col)
    _check_flags(g, dict(preflag=cl["preflag"], flag=flag, near=cl["near"]))
    h2 = c.model == 1
    np.testing.assert_allclose(g["hfilm"][h2], cl["hfilm"][h2],
                               rtol=1e-5 if dtype != M.F64 else 1e-12)


@pytest.mark.parametrize("dtype", DTYPES)
def test_cell_order_matches_grid_convention(dtype):
    # the permutation of the first neighbour stage alone, against the cell
    # ordering the input generator uses (same grid, keys, stable sort)
    c = C.random_cloud(20000, seed=9, h_lo=0.05, h_hi=0.08)
    ctx = M.Context(c.n)
    rd = M.real_dtype(dtype)
    order = torch.empty(c.n, dtype=torch.int32, device="cuda")
    M.cell_order(ctx, torch.tensor(c.pos_h, dtype=rd, device="cuda"), order, dtype)
    np.testing.assert_array_equal(order.cpu().numpy(), C.cell_order(c.pos_h))
    assert ctx.status()["cells_identity"] == 0
    s = C.cell_sorted(c)
    M.cell_order(ctx, torch.tensor(s.pos_h, dtype=rd, device="cuda"), order, dtype)
    np.testing.assert_array_equal(order.cpu().numpy(), np.arange(c.n))
    assert ctx.status()["cells_identity"] == 1
    ctx.close()


def test_neighbours_past_one_scan_chunk(orc):
    # 4.6M rows: more than 1024 scan tiles of 4096 rows, so the tile-sum scan
    # takes several chunks and every warp of its block holds live tiles
    c = C.random_cloud(4_600_000, seed=5, h_lo=0.018, h_hi=0.022, frac2d=0.0)
    rp, col = orc.neighbours(c.pos_h)
    ctx = M.Context(c.n)
    t = torch.tensor(c.pos_h, device="cuda")
    g_rp, g_col, _ = M.neighbours(ctx, t, cap_nnz=int(rp[-1]) + 1024)
    np.testing.assert_array_equal(g_rp.cpu().numpy(), rp)
    np.testing.assert_array_equal(g_col.cpu().numpy(), col)
    ctx.close()


@pytest.mark.parametrize("dtype", DTYPES)
def test_neighbour_edge_cases(orc, dtype):
    ctx = M.Context(64)
    rd = M.real_dtype(dtype)
    cases = [
        np.array([[0, 0, 0, 0.5], [0.5, 0, 0, 0.5], [0, 0.75, 0, 1.0], [2, 2, 2, 0.25]]),
        np.array([[1.0, 2.0, 3.0, 0.1]]),                    # single particle
        np.tile([[0.3, 0.3, 0.3, 0.01]], (40, 1)),            # coincident
        np.array([[0, 0, 0, 1.0], [1e-3, 0, 0, 1.0]]) + 1e3,  # far from the origin
    ]
    for P in cases:
        P = P.astype(np.float32).astype(np.float64)
        rp, col = orc.neighbours(P)
        t = torch.tensor(P, dtype=rd, device="cuda")
        g_rp, g_col, _ = M.neighbours(ctx, t, dtype=dtype)
        np.testing.assert_array_equal(g_rp.cpu().numpy(), rp)
        np.testing.assert_array_equal(g_col.cpu().numpy(), col)
    # empty cloud
    t = torch.zeros((0, 4), dtype=rd, device="cuda")
    g_rp, g_col, _ = M.neighbours(ctx, t, dtype=dtype)
    assert g_rp.cpu().tolist() == [0] and g_col.numel() == 0


def test_boundary_band_pairs_fp32(orc):
    # pairs placed within a few ulps of |x_j - x_i| = (h_i + h_j)/2: the FP32
    # path retakes them in FP64 and must agree with the oracle's definition
    rng = np.random.default_rng(7)
    pts = []
    for k in range(512):
        h = rng.uniform(0.05, 0.2)
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        # pairs on a lattice of spacing 0.6 > max support radius, so pairs are separate
        base = np.array([k % 8, (k // 8) % 8, k // 64]) * 0.6 + rng.uniform(0, 0.1, 3)
        r = h * (1.0 + rng.integers(-3, 4) * 6e-8)
        pts.append([*base, h])
        pts.append([*(base + d * r), h])
    P = np.array(pts).astype(np.float32).astype(np.float64)   # both sides see these values
    rp, col = orc.neighbours(P)
    near = [k for k in range(0, len(P), 2)
            if abs(np.sum((P[k, :3] - P[k + 1, :3]) ** 2) / (P[k, 3] ** 2) - 1) < 1e-5]
    assert len(near) > 100      # most pairs sit inside the FP64 retake band
    ctx = M.Context(P.shape[0])
    g_rp, g_col, _ = M.neighbours(ctx, torch.tensor(P, dtype=torch.float32, device="cuda"))
    np.testing.assert_array_equal(g_rp.cpu().numpy(), rp)
    np.testing.assert_array_equal(g_col.cpu().numpy(), col)


@pytest.mark.parametrize("dtype", DTYPES)
def test_shallow_cylinder_detection(orc, dtype):
    c = C.shallow_layer(dx=0.05, depth_layers=3, extent=1.0, cylinder=True, h_factor=6.0)
    o = _oracle_all(orc, c)
    assert (o["flag"] == 1).sum() > 1000
    g, *_ = run_gpu(c, dtype)
    _check_csr(g, o)
    _check_flags(g, o)
    w = (c.model == 0) & (c.ptype == 2)
    rel = 1e-4 if dtype != M.F64 else 1e-10
    np.testing.assert_allclose(g["eig"][w, 3], o["eig"][w, 3], rtol=rel, atol=rel)
    # |n . w3| agrees (eigenvector sign is arbitrary)
    gn = np.abs(np.sum(g["frame"][w, 4:7] * c.normal[w, :3], 1))
    on = np.abs(np.sum(o["frame"][w, 4:7] * c.normal[w, :3], 1))
    np.testing.assert_allclose(gn, on, atol=1e-4 if dtype != M.F64 else 1e-9)


@pytest.mark.parametrize("dtype", DTYPES)
def test_film_to_bulk_detection(orc, dtype):
    f = C.flat_film(0.01, 0.6, 0.003)
    rp, col = orc.neighbours(f.pos_h)
    cl = orc.classify(f.pos_h, f.model, f.ptype, f.normal, f.vol, f.h3d, f.user, rp, col)
    f.h3d[:] = np.float32(np.median(cl["hfilm"]))     # about half the film transitions
    o = _oracle_all(orc, f)
    assert 0 < (o["flag"] == 2).sum() < f.n
    g, *_ = run_gpu(f, dtype)
    _check_flags(g, o)
    np.testing.assert_allclose(g["hfilm"], o["hfilm"], rtol=1e-5 if dtype != M.F64 else 1e-12)


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("scatter", [False, True])
def test_apply_transpose(orc, dtype, scatter):
    # adjoint identity <apply(f), g> = <f, apply_T(g)> on the GPU's own
    # stencils, and apply_T against the oracle's transpose of its own stencils;
    # gathered through the transpose map, or scattered with atomics (no map)
    c = C.config_small()
    o = _oracle_all(orc, c)
    g, pipe, d, ctx = run_gpu(c, dtype)
    n = c.n
    rp, col = pipe.csr(n)
    tloc = None
    if not scatter:
        tloc = torch.empty(col.numel(), dtype=torch.int16, device="cuda")
        M.transpose_map(ctx, rp, col, tloc)
    rng = np.random.default_rng(3)
    G = rng.normal(size=(n, 4, 4))
    rd = M.real_dtype(dtype)
    gt = torch.tensor(G, dtype=rd, device="cuda")
    gf = torch.full((n, 4), 7.0, dtype=rd, device="cuda")   # overwritten by both forms
    M.apply_ops_backward(ctx, rp, col, tloc, pipe.coef, gt, gf, dtype)
    torch.cuda.synchronize()
    got = gf.double().cpu().numpy()
    lhs = float(np.sum(g["out"] * G))
    rhs = float(np.sum(c.vp.astype(np.float64) * got))
    assert abs(lhs - rhs) <= (1e-5 if dtype != M.F64 else 1e-11) * np.sum(np.abs(g["out"] * G))
    want = orc.apply_T(o["row_ptr"], o["col"], o["coef"], G)
    scale = np.abs(want).max(0)
    assert np.all(np.abs(got - want).max(0) <= TOL[dtype] * scale)


@pytest.mark.parametrize("g3,g2,ga,gc", [(8, 4, 4, 1), (8, 4, 4, 2), (16, 16, 16, 4),
                                         (32, 8, 8, 16)])
def test_launch_shapes_agree_with_oracle(orc, g3, g2, ga, gc):
    c = C.config_small()
    o = _oracle_all(orc, c)
    ctx = M.Context(c.n)
    ctx.set_tuning(stencil3d_group=g3, stencil2d_group=g2, apply_group=ga, classify_group=gc)
    g, *_ = run_gpu(c, M.F32_REFINED, ctx=ctx)
    _check_flags(g, o)
    err, _ = stencil_rowwise_error_vec(o["row_ptr"], g["coef"], o["coef"])
    assert np.all(err <= TOL[M.F32_REFINED]), err
    nw, p99 = column_error(g["out"], o["out"])
    assert np.all(nw <= TOL[M.F32_REFINED]), (nw, p99)
    for bad in (0, 3, 32):
        with pytest.raises(M.MafpError):
            ctx.set_tuning(classify_group=bad)


@pytest.mark.parametrize("pct", [100, 115, 130, 200])
def test_cell_tile_shapes_give_the_oracle_lists(orc, pct):
    """Every cell edge of the neighbour grid (cell_edge_pct, the autotuner's cell
    tile) gives the oracle's neighbour lists bit for bit, in cell order and
    unsorted (cells whose candidate union overflows the mask tile take the
    warp-per-particle path)."""
    for c in (C.cell_sorted(C.config_small()), C.random_cloud(3000, 11)):
        rp, col = orc.neighbours(c.pos_h)
        ctx = M.Context(c.n)
        ctx.set_tuning(cell_edge_pct=pct)
        g, *_ = run_gpu(c, M.F32_REFINED, ctx=ctx, stages=("nbr",))
        assert g["status_block"]["code"] == 0
        np.testing.assert_array_equal(g["row_ptr"], rp)
        np.testing.assert_array_equal(g["col"], col)
        h = float(c.pos_h[:, 3].max())
        assert g["status_block"]["cell_size"] >= pct / 100.0 * h
        ctx.close()
    ctx = M.Context(16)
    for bad in (99, 201):
        with pytest.raises(M.MafpError):
            ctx.set_tuning(cell_edge_pct=bad)
    ctx.close()
