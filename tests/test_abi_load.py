"""The C-ABI library builds for sm_103a, loads without a GPU and exports every
function include/*.h declares (no compute calls here)."""
import ctypes
import glob
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        names |= set(re.findall(r"^\s*(?:int|void|const char \*)\s*(mafp_\w+)\s*\(", src, re.M))
    return sorted(names)


@pytest.fixture(scope="module")
def libpath():
    from paper_2405_13165_gb300 import build
    if not os.path.exists(build.NVCC):
        pytest.skip("nvcc not available")
    return build.build()


def test_header_declares_the_pipeline_calls():
    names = _declared()
    for call in ("mafp_build_neighbours", "mafp_classify_pca", "mafp_build_stencils",
                 "mafp_apply_ops", "mafp_remap_switched", "mafp_apply_ops_backward",
                 "mafp_build_stencils_backward", "mafp_create", "mafp_destroy"):
        assert call in names


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r" T (mafp_\w+)", out))
    missing = [s for s in _declared() if s not in exported]
    assert not missing, missing
    lib = ctypes.CDLL(libpath)
    for s in _declared():
        assert hasattr(lib, s)


def test_defaults_and_host_side_errors(libpath):
    from paper_2405_13165_gb300 import mafp as M
    p = M.default_params()
    assert p.eps_lambda_max == 0.15 and abs(p.theta_star - 0.5235987755982988) < 1e-15
    L = M.lib()
    assert L.mafp_create(None, None, 10, 10) == M.EINVAL
    h = ctypes.c_void_p()
    assert L.mafp_create(ctypes.byref(h), None, 0, 10) == M.EINVAL
    assert L.mafp_build_neighbours(None, 1, 0, None, None, None, 0, None, None, None) == M.EINVAL
    assert L.mafp_destroy(None) == M.OK
    assert L.mafp_last_error(None) == b"null context"
