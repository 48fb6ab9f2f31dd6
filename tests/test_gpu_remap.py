"""GPU parity of the model transition (Sec. 5, Algs. 3 and 4) through the C ABI:
the GPU path detects, smooths and remaps with its own neighbour lists and
flags; the oracle does the same on its own.  Integer outputs (count, old2new,
model, type, last) must be identical; real outputs agree within the rounding
of the precision; total mass is conserved."""
import numpy as np
import pytest

from paper_2405_13165_gb300 import clouds as C

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import oracle as O  # noqa: E402
from paper_2405_13165_gb300 import mafp as M  # noqa: E402
from parity_util import run_gpu  # noqa: E402

KEYS_F4 = ("pos_h", "vp", "normal")
KEYS_F1 = ("rho", "eta", "mass", "diam", "hfilm", "h3d")


def _gpu_remap(c, dtype, cap_factor=4):
    g, pipe, d, ctx = run_gpu(c, dtype, stages=("nbr", "cls"))
    n = c.n
    rd = M.real_dtype(dtype)
    st_in = {k: d[k] for k in KEYS_F4 + KEYS_F1}
    st_in.update(model=d["model"], type=d["ptype"], last=d["last"])
    # the film height the 2D -> 3D transition uses is the state's H
    cap = cap_factor * n + 64
    st_out = {k: torch.zeros((cap,) + tuple(v.shape[1:]), dtype=v.dtype, device="cuda")
              for k, v in st_in.items()}
    old2new = torch.empty(n, dtype=torch.int32, device="cuda")
    n_out = torch.zeros(1, dtype=torch.int64, device="cuda")
    rp, col = pipe.csr(n)
    ctx.reset_status()
    M.remap_switched(ctx, n, st_in, pipe.flag[:n], rp, col, st_out, cap, old2new, n_out, dtype)
    torch.cuda.synchronize()
    status = ctx.status()
    k = int(n_out.item())
    out = {key: v[:k].double().cpu().numpy() if v.dtype in (torch.float32, torch.float64)
           else v[:k].cpu().numpy() for key, v in st_out.items()}
    return g, out, old2new.cpu().numpy(), k, status


def _oracle_remap(c):
    rp, col = O.neighbours(c.pos_h)
    cl = O.classify(c.pos_h, c.model, c.ptype, c.normal, c.vol, c.h3d, c.user, rp, col)
    flag = O.smooth(c.model, cl["preflag"], c.last, rp, col)
    out, o2n, n_out = O.remap(O.cloud_state(c), flag, rp, col)
    return flag, cl["near"], out, o2n, n_out


def _compare(c, dtype, tol, cap_factor=4):
    flag, near, oo, o2n, n_out = _oracle_remap(c)
    assert near.sum() == 0
    g, go, g_o2n, g_n, status = _gpu_remap(c, dtype, cap_factor)
    np.testing.assert_array_equal(g["flag"], flag)
    assert status["code"] == 0 and g_n == n_out == status["n_out"]
    np.testing.assert_array_equal(g_o2n, o2n)
    for k in ("model", "last"):
        np.testing.assert_array_equal(go[k], oo[k])
    np.testing.assert_array_equal(go["type"], oo["ptype"])
    for k in KEYS_F4 + KEYS_F1:
        # normwise per component: averages of mixed-sign values can be near zero
        a, b = go[k], oo[k]
        scale = np.abs(b).max(axis=0)
        assert np.all(np.abs(a - b) <= tol * scale), (k, np.max(np.abs(a - b) / np.maximum(scale, 1e-300)))
    m_in = c.mass.astype(np.float64).sum()
    assert abs(go["mass"].sum() - m_in) <= (1e-5 if dtype != M.F64 else 1e-12) * m_in
    return flag


@pytest.mark.parametrize("dtype", [M.F32_REFINED, M.F64])
def test_remap_3d_to_2d_shallow_cylinder(dtype):
    c = C.shallow_layer(dx=0.05, depth_layers=3, extent=1.0, cylinder=True, h_factor=6.0)
    flag = _compare(c, dtype, 2e-6 if dtype != M.F64 else 1e-12)
    assert (flag == 1).sum() > 1000


@pytest.mark.parametrize("dtype", [M.F32_REFINED, M.F64])
def test_remap_2d_to_3d_thick_film(dtype):
    f = C.flat_film(0.01, 0.5, 0.003)
    rp, col = O.neighbours(f.pos_h)
    cl = O.classify(f.pos_h, f.model, f.ptype, f.normal, f.vol, f.h3d, f.user, rp, col)
    # the 3D resolution set inside the widest gap of the film heights near their
    # 30th percentile: about 70 % of the film transitions, none near the threshold
    hs = np.sort(cl["hfilm"])
    lo, hi = int(0.25 * f.n), int(0.35 * f.n)
    k = lo + int(np.argmax(np.diff(hs[lo:hi + 1])))
    f.h3d[:] = np.float32(0.5 * (hs[k] + hs[k + 1]))
    f.hfilm[:] = np.float32(1.2 * f.h3d[0])        # gamma = ceil(1.2 * 3.5) = 5 per particle
    flag = _compare(f, dtype, 2e-6 if dtype != M.F64 else 1e-12, cap_factor=8)
    assert (flag == 2).sum() > 100


@pytest.mark.parametrize("dtype", [M.F32_REFINED, M.F64])
def test_remap_both_directions_with_user_criterion(dtype):
    # cube on a sheet: a user criterion sends a patch of film to 3D and the
    # shallow bottom of the cube would go to 2D only with its own criteria
    c = C.cube_on_sheet(0.02)
    x = c.pos_h[:, 0].astype(np.float64)
    y = c.pos_h[:, 1].astype(np.float64)
    patch = (c.model == 1) & (np.hypot(x - 0.15, y - 0.15) < 0.08)
    c.user[patch] = C.USER_TO_3D
    c.hfilm[patch] = np.float32(0.05)
    flag = _compare(c, dtype, 2e-6 if dtype != M.F64 else 1e-12)
    assert (flag == 2).sum() > 10


def test_remap_capacity_error_reported():
    f = C.flat_film(0.01, 0.3, 0.003)
    f.user[:] = C.USER_TO_3D
    f.hfilm[:] = np.float32(0.2)
    g, pipe, d, ctx = run_gpu(f, M.F32_REFINED, stages=("nbr", "cls"))
    n = f.n
    st_in = {k: d[k] for k in KEYS_F4 + KEYS_F1}
    st_in.update(model=d["model"], type=d["ptype"], last=d["last"])
    cap = n + 10           # far too small for gamma new particles per film particle
    st_out = {k: torch.zeros((cap,) + tuple(v.shape[1:]), dtype=v.dtype, device="cuda")
              for k, v in st_in.items()}
    old2new = torch.empty(n, dtype=torch.int32, device="cuda")
    n_out = torch.zeros(1, dtype=torch.int64, device="cuda")
    rp, col = pipe.csr(n)
    ctx.reset_status()
    M.remap_switched(ctx, n, st_in, pipe.flag[:n], rp, col, st_out, cap, old2new, n_out,
                     M.F32_REFINED)
    torch.cuda.synchronize()
    st = ctx.status()
    assert st["code"] == M.ECAPACITY and st["required"] == int(n_out.item()) > cap
    assert torch.all(st_out["mass"] == 0)          # nothing written
