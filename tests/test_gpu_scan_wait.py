"""The bounded device-side wait of the one-pass scan (tiles wait for the
prefix of earlier tiles).  With params.wait_limit = 0 a tile that finds an
earlier tile's prefix not yet published gives up at once: the call's status
block records MAFP_ETIMEOUT and nothing waits longer.  The scan's tile states
and tickets are left clean after such a call, so the same context keeps
running, and a context with the default limit builds the oracle's lists."""
import numpy as np
import pytest

from paper_2405_13165_gb300 import clouds as C

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import oracle as O  # noqa: E402
from paper_2405_13165_gb300 import mafp as M  # noqa: E402


def _build(ctx, pos, n):
    row_ptr = torch.zeros(n + 1, dtype=torch.int64, device="cuda")
    col = torch.empty(200 * n, dtype=torch.int32, device="cuda")
    ctx.reset_status()
    M.build_neighbours(ctx, pos, row_ptr, col)
    torch.cuda.synchronize()
    return ctx.status(), row_ptr, col


def test_zero_wait_limit_times_out_and_the_context_recovers():
    c = C.cell_sorted(C.jet_on_plate(None, n_target=400_000))
    n = c.n
    pos = torch.from_numpy(c.pos_h).cuda()
    ctx0 = M.Context(n, params=M.default_params(wait_limit=0))
    codes = []
    for _ in range(5):
        st, _, _ = _build(ctx0, pos, n)
        codes.append(st["code"])
        if st["code"] == M.ETIMEOUT:
            break
    # ~100 tiles start together: some tile meets an unpublished predecessor
    assert M.ETIMEOUT in codes, codes
    assert all(cd in (0, M.ETIMEOUT) for cd in codes), codes
    # later calls of the same context still run to the end (states were cleared)
    small = C.config_small()
    st, _, _ = _build(ctx0, torch.from_numpy(small.pos_h).cuda(), small.n)
    assert st["code"] in (0, M.ETIMEOUT), st
    ctx0.close()
    # the default limit: the oracle's lists
    ctx1 = M.Context(n)
    st, row_ptr, col = _build(ctx1, pos, n)
    assert st["code"] == 0, st
    rp, oc = O.neighbours(c.pos_h)
    np.testing.assert_array_equal(row_ptr.cpu().numpy(), rp)
    np.testing.assert_array_equal(col[: rp[-1]].cpu().numpy(), oc)
    ctx1.close()
