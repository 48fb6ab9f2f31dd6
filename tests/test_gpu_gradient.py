"""GPU gradients through the C ABI: the transpose of apply_ops (fields) and the
stencil adjoint (positions), against the FP64 oracle gradient (itself pinned by
central finite differences) and, in FP64, against finite differences of the
GPU forward.  Film rows take their tangent frame from the local PCA of the
positions, so every forward evaluated at moved positions recomputes the frame
(classify) first; flat, tilted and curved films are covered."""
import numpy as np
import pytest

from paper_2405_13165_gb300 import clouds as C

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import oracle as O  # noqa: E402
from paper_2405_13165_gb300 import mafp as M  # noqa: E402
from paper_2405_13165_gb300.autograd import gfdm_operators  # noqa: E402
from parity_util import run_gpu  # noqa: E402
from grad_shapes import SHAPES, shape  # noqa: E402


def _setup(c, dtype):
    g, pipe, d, ctx = run_gpu(c, dtype, stages=("nbr", "cls"))
    n = c.n
    rp, col = pipe.csr(n)
    return ctx, d, rp, col, pipe.frame[:n].clone()


def frame_of(ctx, d, pos, rp, col, dtype):
    """The tangent frames classify computes at positions `pos` (neighbour sets
    held fixed), as a forward at moved positions needs them."""
    n = pos.shape[0]
    rd = M.real_dtype(dtype)
    u8 = lambda: torch.empty(n, dtype=torch.uint8, device="cuda")
    frame = torch.empty(n, 8, dtype=rd, device="cuda")
    M.classify_pca(ctx, pos.contiguous(), d["model"], d["ptype"], d["normal"], d["vol"], d["h3d"],
                   d["user"], d["last"], rp, col, u8(), u8(),
                   torch.empty(n, 4, dtype=rd, device="cuda"), frame,
                   torch.empty(n, dtype=rd, device="cuda"), None, dtype)
    return frame


@pytest.mark.parametrize("shape_name", SHAPES)
@pytest.mark.parametrize("dtype", [M.F32_REFINED, M.F64])
@pytest.mark.parametrize("loss", ["laplacian", "random"])
def test_position_gradient_matches_oracle(dtype, loss, shape_name):
    c = (C.cube_on_sheet(0.04, cube=0.32, sheet=1.0) if shape_name == "flat"
         else shape(shape_name)[0])
    ctx, d, rp, col, frame = _setup(c, dtype)
    pos = d["pos_h"].clone().requires_grad_(True)
    fields = d["fields"].clone().requires_grad_(True)
    out = gfdm_operators(ctx, pos, fields, rp, col, d["model"], frame, dtype)
    rng = np.random.default_rng(4)
    Gr = rng.normal(size=(c.n, 4, 4))
    if loss == "laplacian":
        L = (out[:, :, 3] ** 2).sum()
    else:
        L = (out * torch.tensor(Gr, dtype=out.dtype, device="cuda")).sum()
    L.backward()
    gpos = pos.grad.double().cpu().numpy()
    gfld = fields.grad.double().cpu().numpy()
    # oracle on its own neighbours / stencils
    P = c.pos_h.astype(np.float64)
    orp, ocol = O.neighbours(P)
    coef, status, _ = O.stencils(P, c.model, orp, ocol)
    oout = O.apply(orp, ocol, coef, c.vp)
    if loss == "laplacian":
        G = np.zeros_like(oout)
        G[:, :, 3] = 2.0 * oout[:, :, 3]
    else:
        G = Gr
    og = O.stencil_grad(P, c.model, orp, ocol, c.vp, G)
    ogf = O.apply_T(orp, ocol, coef, G)
    tol = 2e-3 if dtype != M.F64 else 1e-8
    scale = np.abs(og[:, :3]).max(0)
    assert np.all(np.abs(gpos[:, :3] - og[:, :3]).max(0) <= tol * scale), \
        (np.abs(gpos[:, :3] - og[:, :3]).max(0) / scale)
    assert np.all(gpos[:, 3] == 0)
    fscale = np.abs(ogf).max(0)
    assert np.all(np.abs(gfld - ogf).max(0) <= tol * fscale), np.abs(gfld - ogf).max(0) / fscale
    ctx.close()


@pytest.mark.parametrize("shape_name", ["flat", "tilted"])
def test_gradcheck_fp64_tiny_cloud(shape_name):
    # FP64 forward and hand-written backward agree with torch's finite
    # differences; the forward recomputes the film frames from the positions
    c = C.cube_on_sheet(0.1, cube=0.5, sheet=1.0)        # 125 + 75 particles
    if shape_name == "tilted":
        c = C.rotated(c, (1.0, 0.4, 0.2), 0.6)
    ctx, d, rp, col, frame = _setup(c, M.F64)
    pos = d["pos_h"].clone().requires_grad_(True)
    fields = d["fields"].clone().requires_grad_(True)

    def f(p, u):
        # only x, y, z carry gradients; h enters as a constant
        full = torch.cat([p, d["pos_h"][:, 3:]], 1).contiguous()
        fr = frame_of(ctx, d, full.detach(), rp, col, M.F64)
        return gfdm_operators(ctx, full, u, rp, col, d["model"], fr, M.F64)

    xyz = pos[:, :3].detach().clone().requires_grad_(True)
    assert torch.autograd.gradcheck(f, (xyz, fields), eps=1e-7, atol=1e-6, rtol=1e-5,
                                    nondet_tol=1e-9, fast_mode=True)
    ctx.close()


@pytest.mark.parametrize("shape_name", SHAPES)
def test_fp64_film_gradient_matches_central_differences(shape_name):
    """Every coordinate of film particles, FP64 GPU adjoint against central
    differences of the FP64 GPU forward (frames recomputed at every point)."""
    c, dx = shape(shape_name)
    ctx, d, rp, col, frame = _setup(c, M.F64)
    n = c.n
    rng = np.random.default_rng(8)
    G = torch.tensor(rng.normal(size=(n, 4, 4)), dtype=torch.float64, device="cuda")
    coef = torch.empty(col.numel(), 4, dtype=torch.float64, device="cuda")
    status = torch.empty(n, dtype=torch.uint8, device="cuda")
    cond = torch.empty(n, dtype=torch.float32, device="cuda")
    out = torch.empty(n, 4, 4, dtype=torch.float64, device="cuda")

    def loss(pos):
        fr = frame_of(ctx, d, pos, rp, col, M.F64)
        M.build_stencils(ctx, pos, d["model"], fr, rp, col, coef, status, cond, M.F64)
        M.apply_ops(ctx, rp, col, coef, d["fields"], out, M.F64)
        return float((out * G).sum().item())

    pos = d["pos_h"].clone()
    gpos = torch.empty_like(pos)
    M.build_stencils_backward(ctx, pos, d["model"], frame, rp, col, d["fields"], G, gpos, M.F64)
    g = gpos.cpu().numpy()
    P = c.pos_h.astype(np.float64)
    rpn, coln = rp.cpu().numpy(), col.cpu().numpy()
    step = 1e-4 * dx
    film = np.nonzero(c.model == 1)[0]
    checked = 0
    for k in rng.permutation(film):
        r = coln[rpn[k]:rpn[k + 1]]
        dist = np.linalg.norm(P[r, :3] - P[k, :3], axis=1)
        if np.any(np.abs(dist - 0.5 * (P[r, 3] + P[k, 3])) <= 10 * step):
            continue
        for a in (0, 1, 2):
            def central(st):
                pp, pm = pos.clone(), pos.clone()
                pp[k, a] += st
                pm[k, a] -= st
                return (loss(pp) - loss(pm)) / (2 * st)
            fd = (4.0 * central(step / 2) - central(step)) / 3.0
            scale = max(abs(fd), 1e-3 * np.abs(g[:, :3]).max())
            assert abs(g[k, a] - fd) <= 1e-5 * scale + 1e-9, (shape_name, k, a, g[k, a], fd)
            checked += 1
        if checked >= 45:
            break
    assert checked >= 45
    ctx.close()


@pytest.mark.parametrize("dtype", [M.F32_REFINED, M.F64])
def test_adjoint_launch_shapes_agree_with_oracle(dtype):
    """Every grad3d_group / grad2d_group (lanes per 3D / film particle of the
    position adjoint) gives the oracle's gradient; in FP64 the 2- and 4-lane 3D
    choices run the 8-lane kernel."""
    c = C.cube_on_sheet(0.04, cube=0.32, sheet=1.0)
    ctx, d, rp, col, frame = _setup(c, dtype)
    rng = np.random.default_rng(11)
    Gr = rng.normal(size=(c.n, 4, 4))
    P = c.pos_h.astype(np.float64)
    orp, ocol = O.neighbours(P)
    og = O.stencil_grad(P, c.model, orp, ocol, c.vp, Gr)
    scale = np.abs(og[:, :3]).max(0)
    tol = 2e-3 if dtype != M.F64 else 1e-8
    gout = torch.tensor(Gr, dtype=d["pos_h"].dtype, device="cuda").contiguous()
    gpos = torch.empty_like(d["pos_h"])
    for gb, gf in ((2, 1), (2, 2), (4, 2), (8, 4), (16, 8), (32, 16)):
        ctx.set_tuning(grad3d_group=gb, grad2d_group=gf)
        assert ctx.tuning()["grad3d_group"] == gb and ctx.tuning()["grad2d_group"] == gf
        gpos.fill_(float("nan"))
        M.build_stencils_backward(ctx, d["pos_h"], d["model"], frame, rp, col, d["fields"],
                                  gout, gpos, dtype)
        got = gpos.double().cpu().numpy()
        err = np.abs(got[:, :3] - og[:, :3]).max(0)
        assert np.all(err <= tol * scale), (gb, err / scale)
        assert np.all(got[:, 3] == 0)
    with pytest.raises(M.MafpError):
        ctx.set_tuning(grad3d_group=1)
    with pytest.raises(M.MafpError):
        ctx.set_tuning(grad2d_group=32)
    ctx.close()
