"""mafp_build_stencils_noalloc: the allocation-free stencil build.

Callers that cannot allocate device memory (a plug-in whose host application
owns the device-memory budget, or a time step that must not stall on the
implicit synchronisation of cudaMalloc / cudaFree) use this entry point; its
only scratch is an array compiled into the library: the queue of rows redone
in FP64.  This test calls it through the C ABI several times in a row and
checks every result against the context-based mafp_build_stencils and against
the FP64 oracle, within the stencil tolerance of the parity tests:
  - with the FP64 threshold cond_fp64 = 1 every FP32 row is queued into the
    static array and redone in FP64 (status MAFP_STENCIL_FP64), twice in a row;
  - a third call with the default threshold queues (almost) nothing, so a queue
    length left over from the calls before would redo rows it should not and
    show up in their status.
Kept in its own file, collected last.
"""
import ctypes as C

import numpy as np
import pytest

from paper_2405_13165_gb300 import clouds as CL

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import oracle as O  # noqa: E402
from paper_2405_13165_gb300 import mafp as M  # noqa: E402
from parity_util import TOL, run_gpu, stencil_rowwise_error_vec  # noqa: E402


def _noalloc(n, dtype, params, d, frame, row_ptr, col, coef, status, cond):
    L = M.lib()
    fn = L.mafp_build_stencils_noalloc
    p = C.c_void_p
    fn.argtypes = [C.c_int64, C.c_int32, p, p, p, p, p, p, p, p, p, p]
    fn.restype = C.c_int
    return fn(n, dtype, C.cast(C.byref(params), p), p(d["pos_h"].data_ptr()),
              p(d["model"].data_ptr()), p(frame.data_ptr()), p(row_ptr.data_ptr()),
              p(col.data_ptr()), p(coef.data_ptr()), p(status.data_ptr()), p(cond.data_ptr()),
              p(torch.cuda.current_stream().cuda_stream))


@pytest.mark.parametrize("dtype", [M.F32_REFINED, M.F64])
def test_noalloc_matches_context_entry_point_and_oracle(dtype):
    c = CL.config_small()
    n = c.n
    orp, ocol = O.neighbours(c.pos_h)
    ocoef, ostatus, _ = O.stencils(c.pos_h, c.model, orp, ocol)
    for call, cond_fp64 in enumerate((1.0, 1.0, 1e4)):
        prm = M.default_params(cond_fp64=cond_fp64)
        ctx = M.Context(n, params=prm)
        # context path: neighbours, frames, stencils with the same threshold
        g, pipe, d, _ = run_gpu(c, dtype, ctx=ctx)
        row_ptr, col = pipe.csr(n)
        np.testing.assert_array_equal(g["col"], ocol)
        frame = pipe.frame[:n]
        coef = torch.full_like(pipe.coef[: col.numel()], float("nan"))
        status = torch.full((n,), 255, dtype=torch.uint8, device="cuda")
        cond = torch.zeros(n, dtype=torch.float32, device="cuda")
        rc = _noalloc(n, dtype, prm, d, frame, row_ptr, col, coef, status, cond)
        assert rc == M.OK, (call, rc)
        torch.cuda.synchronize()
        st = status.cpu().numpy()
        np.testing.assert_array_equal(st, g["status"])
        ok = ostatus == 0
        assert np.all((st == M.STENCIL_DEFICIENT) == ~ok)
        if dtype == M.F64:
            assert np.all(st[ok] == M.STENCIL_OK)
        elif cond_fp64 == 1.0:
            # every row went through the queue in the static array and its FP64 redo
            assert np.all(st[ok] == M.STENCIL_FP64), (call, np.bincount(st))
        else:
            # the queue starts empty again: only rows above the default threshold
            assert np.sum(st == M.STENCIL_FP64) < 0.01 * n, (call, np.bincount(st))
        a = coef.double().cpu().numpy()
        err, _ = stencil_rowwise_error_vec(g["row_ptr"], a, g["coef"])
        assert np.all(err <= TOL[dtype]), (call, err)
        err, _ = stencil_rowwise_error_vec(orp, a, ocoef)
        assert np.all(err <= TOL[dtype]), (call, err)
        ctx.close()


def test_noalloc_rejects_too_many_particles():
    L = M.lib()
    fn = L.mafp_build_stencils_noalloc
    fn.argtypes = [C.c_int64, C.c_int32] + [C.c_void_p] * 10
    fn.restype = C.c_int
    too_many = (1 << 20) + 1
    assert fn(too_many, M.F32_REFINED, *([None] * 10)) == M.ECAPACITY
