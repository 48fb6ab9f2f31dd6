"""Batches of independent clouds through mafp_build_neighbours_batched and the
rest of the pipeline: the result over the batch equals, cloud by cloud, the
oracle run on each cloud alone (clouds overlap in space, so any neighbour that
crossed a cloud boundary would show), plus offsets edge cases and CUDA-graph
replay of the whole batched pass."""
import numpy as np
import pytest

from paper_2405_13165_gb300 import clouds as C

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2405_13165_gb300 import mafp as M  # noqa: E402
from paper_2405_13165_gb300.pipeline import Pipeline, cloud_to_device  # noqa: E402
from parity_util import (P99_BAR, TOL, column_error, run_gpu,  # noqa: E402
                         stencil_rowwise_error_vec)

DTYPES = [M.F32_REFINED, M.F64]


def _batch(nclouds, n_lo, n_hi, seed, sort=True):
    parts = C.batched_clouds(nclouds, n_lo, n_hi, seed=seed)
    if sort:
        parts = [C.cell_sorted(c) for c in parts]
    off = np.zeros(len(parts) + 1, np.int64)
    off[1:] = np.cumsum([c.n for c in parts])
    return parts, C.concat(parts), off


def _oracle_batch(orc, parts, off):
    """Per-cloud oracle, stitched into one CSR with global column indices."""
    rps, cols, res = [np.zeros(1, np.int64)], [], {}
    keys = ("flag", "preflag", "near", "status")
    acc = {k: [] for k in keys + ("coef", "out")}
    for b, c in enumerate(parts):
        rp, col = orc.neighbours(c.pos_h)
        cl = orc.classify(c.pos_h, c.model, c.ptype, c.normal, c.vol, c.h3d, c.user, rp, col)
        flag = orc.smooth(c.model, cl["preflag"], c.last, rp, col)
        coef, status, _ = orc.stencils(c.pos_h, c.model, rp, col)
        out = orc.apply(rp, col, coef, c.vp)
        rps.append(rp[1:] + rps[-1][-1])
        cols.append(col + off[b])
        for k, v in (("flag", flag), ("preflag", cl["preflag"]), ("near", cl["near"]),
                     ("status", status), ("coef", coef), ("out", out)):
            acc[k].append(v)
    res = {k: np.concatenate(v) for k, v in acc.items()}
    res["row_ptr"] = np.concatenate(rps)
    res["col"] = np.concatenate(cols).astype(np.int32)
    return res


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("sort", [True, False])
def test_batch_matches_per_cloud_oracle(orc, dtype, sort):
    parts, c, off = _batch(10, 150, 4000, seed=7, sort=sort)
    o = _oracle_batch(orc, parts, off)
    g, *_ = run_gpu(c, dtype, cloud_offset=off)
    assert g["status_block"]["code"] == 0
    np.testing.assert_array_equal(g["row_ptr"], o["row_ptr"])
    np.testing.assert_array_equal(g["col"], o["col"])
    far = o["near"] == 0
    np.testing.assert_array_equal(g["preflag"][far], o["preflag"][far])
    np.testing.assert_array_equal(g["flag"][far], o["flag"][far])
    np.testing.assert_array_equal(g["status"] == M.STENCIL_DEFICIENT, o["status"] == 1)
    err, _ = stencil_rowwise_error_vec(o["row_ptr"], g["coef"], o["coef"])
    assert np.all(err <= TOL[dtype]), err
    nw, p99 = column_error(g["out"], o["out"])
    assert np.all(nw <= TOL[dtype]), (nw, p99)
    assert np.all(p99 <= P99_BAR[dtype]), p99
    # the order output is the concatenation of per-cloud cell orders
    order = g["order"]
    for b in range(len(parts)):
        seg = order[off[b]:off[b + 1]]
        assert seg.min() >= off[b] and seg.max() < off[b + 1]
        if sort:
            np.testing.assert_array_equal(seg, np.arange(off[b], off[b + 1]))


def test_single_cloud_batch_equals_plain_call(orc):
    c = C.cell_sorted(C.config_small())
    a, *_ = run_gpu(c, M.F32_REFINED, stages=("nbr",))
    b, *_ = run_gpu(c, M.F32_REFINED, stages=("nbr",), cloud_offset=np.array([0, c.n]))
    np.testing.assert_array_equal(a["row_ptr"], b["row_ptr"])
    np.testing.assert_array_equal(a["col"], b["col"])
    assert a["status_block"]["ncells"] == b["status_block"]["ncells"]
    assert a["status_block"]["cell_size"] == b["status_block"]["cell_size"]


def test_empty_clouds_and_identical_copies(orc):
    # empty clouds anywhere in the offsets; two bit-identical copies of a cloud
    # stored back to back must each see only themselves
    c = C.cell_sorted(C.cube_on_sheet(0.05, cube=0.3, sheet=0.8, seed=11))
    both = C.concat([c, c])
    n = c.n
    off = np.array([0, 0, n, n, n, 2 * n, 2 * n])
    rp, col = orc.neighbours(c.pos_h)
    g, *_ = run_gpu(both, M.F32_REFINED, stages=("nbr",), cloud_offset=off)
    assert g["status_block"]["code"] == 0
    np.testing.assert_array_equal(g["row_ptr"], np.concatenate([rp, rp[1:] + rp[-1]]))
    np.testing.assert_array_equal(g["col"], np.concatenate([col, col + n]))


def test_bad_offsets_are_reported():
    c = C.cube_on_sheet(0.05, cube=0.3, sheet=0.8, seed=11)
    n = c.n
    ctx = M.Context(n)
    d = cloud_to_device(c)
    row_ptr = torch.zeros(n + 1, dtype=torch.int64, device="cuda")
    col = torch.full((200 * n,), -7, dtype=torch.int32, device="cuda")
    for off in ([0, n // 2, n - 1], [1, n // 2, n], [0, n // 2 + 5, n // 2, n]):
        ctx.reset_status()
        o = torch.tensor(off, dtype=torch.int64, device="cuda")
        M.build_neighbours_batched(ctx, o, d["pos_h"], row_ptr, col)
        torch.cuda.synchronize()
        assert ctx.status()["code"] == M.EINVAL, off
        assert bool((col == -7).all())
    with pytest.raises(M.MafpError):
        o = torch.zeros(M.MAX_CLOUDS + 2, dtype=torch.int64, device="cuda")
        M.build_neighbours_batched(ctx, o, d["pos_h"], row_ptr, col)
    ctx.close()


def test_many_tiny_clouds(orc):
    # more clouds than bounding-box blocks: one block part per cloud
    parts = [C.random_cloud(int(k), seed=100 + k, h_lo=0.2, h_hi=0.3) for k in
             np.random.default_rng(3).integers(1, 40, size=3000)]
    off = np.zeros(len(parts) + 1, np.int64)
    off[1:] = np.cumsum([p.n for p in parts])
    c = C.concat(parts)
    g, *_ = run_gpu(c, M.F32_REFINED, stages=("nbr",), cloud_offset=off)
    assert g["status_block"]["code"] == 0
    rows = []
    for b in np.random.default_rng(5).choice(len(parts), 200, replace=False):
        rp, col = orc.neighbours(parts[b].pos_h)
        s = g["row_ptr"][off[b]:off[b + 1] + 1]
        np.testing.assert_array_equal(s - s[0], rp)
        np.testing.assert_array_equal(g["col"][s[0]:s[-1]], col + off[b])
        rows.append(b)
    assert rows


def test_graph_replay_of_batched_pass(orc):
    parts, c, off = _batch(6, 300, 3000, seed=9)
    n = c.n
    ctx = M.Context(n)
    pipe = Pipeline(ctx, n, 400 * n, M.F32_REFINED)
    d = cloud_to_device(c, cloud_offset=off)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        pipe.step(d, stream=s)          # eager pass (first-call set-up)
    torch.cuda.synchronize()
    ref = [t.clone() for t in (pipe.row_ptr, pipe.col, pipe.flag, pipe.coef, pipe.out)]
    for t in (pipe.col, pipe.coef, pipe.out):
        t.zero_()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=s):
        pipe.step(d, stream=s)
    for _ in range(2):
        for t in (pipe.col, pipe.coef, pipe.out):
            t.zero_()
        graph.replay()
        torch.cuda.synchronize()
        for a, b in zip(ref, (pipe.row_ptr, pipe.col, pipe.flag, pipe.coef, pipe.out)):
            assert torch.equal(a, b)
    assert ctx.status()["code"] == 0
    ctx.close()


@pytest.fixture(scope="module")
def full_batch():
    c, off = C.config_batched()              # 256 clouds, about 12M particles
    n = c.n
    ctx = M.Context(n)
    pipe = Pipeline(ctx, n, 160 * n, M.F32_REFINED)
    d = cloud_to_device(c, cloud_offset=off)
    ctx.reset_status()
    pipe.step(d)
    torch.cuda.synchronize()
    st = ctx.status()
    yield c, off, pipe, st
    ctx.close()


def test_full_batch_sampled_clouds(orc, full_batch):
    # the full 256-cloud batch; CSR, flags, stencils and outputs of a seeded
    # sample of whole clouds (always the largest and the smallest) vs the oracle
    c, off, pipe, st = full_batch
    assert st["code"] == 0 and st["cells_identity"] == 1
    sizes = np.diff(off)
    pick = set(np.random.default_rng(31).choice(len(sizes), 4, replace=False).tolist())
    pick |= {int(sizes.argmax()), int(sizes.argmin())}
    for b in sorted(pick):
        lo, hi = int(off[b]), int(off[b + 1])
        part = c.take(np.arange(lo, hi))
        rp, col = orc.neighbours(part.pos_h)
        s = pipe.row_ptr[lo:hi + 1].cpu().numpy()
        np.testing.assert_array_equal(s - s[0], rp)
        np.testing.assert_array_equal(pipe.col[s[0]:s[-1]].cpu().numpy(), col + lo)
        cl = orc.classify(part.pos_h, part.model, part.ptype, part.normal, part.vol, part.h3d,
                          part.user, rp, col)
        flag = orc.smooth(part.model, cl["preflag"], part.last, rp, col)
        far = cl["near"] == 0
        np.testing.assert_array_equal(pipe.preflag[lo:hi].cpu().numpy()[far], cl["preflag"][far])
        np.testing.assert_array_equal(pipe.flag[lo:hi].cpu().numpy()[far], flag[far])
        coef, status, _ = orc.stencils(part.pos_h, part.model, rp, col)
        out = orc.apply(rp, col, coef, part.vp)
        gcoef = pipe.coef[s[0]:s[-1]].double().cpu().numpy()
        err, _ = stencil_rowwise_error_vec(rp, gcoef, coef)
        assert np.all(err <= TOL[M.F32_REFINED]), (b, err)
        nw, p99 = column_error(pipe.out[lo:hi].double().cpu().numpy(), out)
        assert np.all(nw <= TOL[M.F32_REFINED]), (b, nw, p99)
        assert np.all(p99 <= P99_BAR[M.F32_REFINED]), (b, p99)
        gstatus = pipe.status[lo:hi].cpu().numpy()
        np.testing.assert_array_equal(gstatus == M.STENCIL_DEFICIENT, status == 1)


def test_full_batch_rows_stay_in_their_cloud(full_batch):
    # property at any size: every column of every row lies in the row's cloud,
    # and every row holds itself exactly once
    c, off, pipe, st = full_batch
    n = c.n
    rp = pipe.row_ptr[: n + 1]
    offt = torch.tensor(off, device="cuda")
    cloud = torch.repeat_interleave(torch.arange(len(off) - 1, device="cuda", dtype=torch.int32),
                                    offt[1:] - offt[:-1])
    step = 1 << 20
    for r0 in range(0, n, step):
        r1 = min(n, r0 + step)
        lens = rp[r0 + 1:r1 + 1] - rp[r0:r1]
        rows = torch.repeat_interleave(torch.arange(r0, r1, device="cuda"), lens)
        cols = pipe.col[int(rp[r0]):int(rp[r1])].long()
        assert torch.equal(cloud[rows], cloud[cols])
        hits = torch.zeros(r1 - r0, dtype=torch.int64, device="cuda")
        hits.index_add_(0, rows[rows == cols] - r0, torch.ones_like(rows[rows == cols]))
        assert bool((hits == 1).all())
