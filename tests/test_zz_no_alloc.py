"""mafp_build_stencils_noalloc: the allocation-free stencil build.

Callers that cannot allocate device memory (a plug-in whose host application
owns the device-memory budget, or a time step that must not stall on the
implicit synchronisation of cudaMalloc / cudaFree) use this entry point; its
only scratch is an array compiled into the library.  This test calls it
through the C ABI twice in a row and checks both results against the
context-based mafp_build_stencils, within the stencil tolerance of the
parity tests.  Kept in its own file, collected last.
"""
import ctypes as C

import numpy as np
import pytest

from paper_2405_13165_gb300 import clouds as CL

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2405_13165_gb300 import mafp as M  # noqa: E402
from parity_util import TOL, run_gpu, stencil_rowwise_error_vec  # noqa: E402


def _noalloc(n, dtype, d, frame, row_ptr, col, coef, status, cond):
    L = M.lib()
    fn = L.mafp_build_stencils_noalloc
    p = C.c_void_p
    fn.argtypes = [C.c_int64, C.c_int32, p, p, p, p, p, p, p, p, p, p]
    fn.restype = C.c_int
    return fn(n, dtype, None, p(d["pos_h"].data_ptr()), p(d["model"].data_ptr()),
              p(frame.data_ptr()), p(row_ptr.data_ptr()), p(col.data_ptr()),
              p(coef.data_ptr()), p(status.data_ptr()), p(cond.data_ptr()),
              p(torch.cuda.current_stream().cuda_stream))


@pytest.mark.parametrize("dtype", [M.F32_REFINED, M.F64])
def test_noalloc_matches_context_entry_point_twice(dtype):
    c = CL.config_small()
    g, pipe, d, ctx = run_gpu(c, dtype)          # context path: neighbours, frames, stencils
    n = c.n
    row_ptr, col = pipe.csr(n)
    frame = pipe.frame[:n]
    for call in range(2):
        coef = torch.full_like(pipe.coef[: col.numel()], float("nan"))
        status = torch.full((n,), 255, dtype=torch.uint8, device="cuda")
        cond = torch.zeros(n, dtype=torch.float32, device="cuda")
        rc = _noalloc(n, dtype, d, frame, row_ptr, col, coef, status, cond)
        assert rc == M.OK, (call, rc)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(status.cpu().numpy(), g["status"])
        err, _ = stencil_rowwise_error_vec(g["row_ptr"], coef.double().cpu().numpy(), g["coef"])
        assert np.all(err <= TOL[dtype]), (call, err)
    ctx.close()


def test_noalloc_rejects_too_many_particles():
    L = M.lib()
    fn = L.mafp_build_stencils_noalloc
    fn.argtypes = [C.c_int64, C.c_int32] + [C.c_void_p] * 10
    fn.restype = C.c_int
    too_many = (1 << 20) + 1
    assert fn(too_many, M.F32_REFINED, *([None] * 10)) == M.ECAPACITY
