"""Device-detected conditions of the neighbour stage, made on the host: a
position or smoothing length that is not finite (or h <= 0) gives
MAFP_ENONFINITE with the count of bad particles, and a column capacity below
nnz gives MAFP_ECAPACITY with the required size and leaves the column array
untouched.  In both cases every kernel after the grid set-up returns without
touching the lists (the grid's ok flag is cleared, or row_ptr[n] > cap_nnz),
and the context builds correct lists again after mafp_reset_status."""
import numpy as np
import pytest

from paper_2405_13165_gb300 import clouds as C

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import oracle as O  # noqa: E402
from paper_2405_13165_gb300 import mafp as M  # noqa: E402
from paper_2405_13165_gb300.pipeline import cloud_to_device  # noqa: E402

SENTINEL = -7


def _build(ctx, pos, cap, dtype):
    n = pos.shape[0]
    row_ptr = torch.zeros(n + 1, dtype=torch.int64, device="cuda")
    col_full = torch.full((cap + 64,), SENTINEL, dtype=torch.int32, device="cuda")
    nnz = torch.zeros(1, dtype=torch.int64, device="cuda")
    ctx.reset_status()
    M.build_neighbours(ctx, pos, row_ptr, col_full[:cap], nnz, None, dtype)
    torch.cuda.synchronize()
    return ctx.status(), row_ptr, col_full, nnz


@pytest.mark.parametrize("dtype", [M.F32_REFINED, M.F64])
@pytest.mark.parametrize("bad", ["nan_x", "inf_z", "zero_h", "nan_h"])
def test_nonfinite_input_is_reported(dtype, bad):
    c = C.config_small()
    n = c.n
    d = cloud_to_device(c, dtype)
    ctx = M.Context(n)
    pos = d["pos_h"].clone()
    rows = [17, 2000, n - 1]
    for r in rows:
        if bad == "nan_x":
            pos[r, 0] = float("nan")
        elif bad == "inf_z":
            pos[r, 2] = float("inf")
        elif bad == "zero_h":
            pos[r, 3] = 0.0
        else:
            pos[r, 3] = float("nan")
    cap = 400 * n
    st, row_ptr, col_full, nnz = _build(ctx, pos, cap, dtype)
    assert st["code"] == M.ENONFINITE, st
    assert st["n_nonfinite"] == len(rows) and st["required"] == len(rows), st
    assert torch.all(col_full == SENTINEL).item()
    # the same context, status cleared, builds the oracle's lists from clean input
    st, row_ptr, col_full, nnz = _build(ctx, d["pos_h"], cap, dtype)
    assert st["code"] == 0 and st["n_nonfinite"] == 0, st
    rp, col = O.neighbours(c.pos_h)
    np.testing.assert_array_equal(row_ptr.cpu().numpy(), rp)
    np.testing.assert_array_equal(col_full[: rp[-1]].cpu().numpy(), col)
    ctx.close()


@pytest.mark.parametrize("dtype", [M.F32_REFINED, M.F64])
@pytest.mark.parametrize("short", [1, 1000])
def test_column_capacity_below_nnz(dtype, short):
    c = C.config_small()
    n = c.n
    d = cloud_to_device(c, dtype)
    ctx = M.Context(n)
    rp, col = O.neighbours(c.pos_h)
    nnz_true = int(rp[-1])
    st, row_ptr, col_full, nnz = _build(ctx, d["pos_h"], nnz_true - short, dtype)
    assert st["code"] == M.ECAPACITY and st["required"] == nnz_true, st
    assert st["nnz"] == nnz_true and int(nnz.item()) == nnz_true
    # row_ptr is still written, col is not
    np.testing.assert_array_equal(row_ptr.cpu().numpy(), rp)
    assert torch.all(col_full == SENTINEL).item()
    # exactly enough room: no error, the oracle's lists
    st, row_ptr, col_full, nnz = _build(ctx, d["pos_h"], nnz_true, dtype)
    assert st["code"] == 0, st
    np.testing.assert_array_equal(col_full[:nnz_true].cpu().numpy(), col)
    assert torch.all(col_full[nnz_true:] == SENTINEL).item()
    ctx.close()
