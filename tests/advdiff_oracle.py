"""The advection-diffusion loop on the CPU: every stage through the FP64
oracle, the time loop's own updates restated in numpy float32 (user criterion,
explicit Euler step, transport, cell-order permutation), and the analytic
solution of the temperature problem."""
import numpy as np

import oracle as O
from paper_2405_13165_gb300 import clouds as C

F32 = np.float32
KEYS_F = ("pos_h", "vp", "normal", "rho", "eta", "mass", "diam", "hfilm", "h3d")
KEYS_U8 = ("model", "ptype", "last")
BAND = (1.0, 2.0)


def initial_state(cloud) -> dict:
    s = {k: np.array(getattr(cloud, k), dtype=F32) for k in KEYS_F}
    s.update({k: np.array(getattr(cloud, k), dtype=np.uint8) for k in KEYS_U8})
    return s


def user_flags(P, model):
    x = P[:, 0]
    inside = (x >= F32(BAND[0])) & (x <= F32(BAND[1]))
    u = np.zeros(model.shape, np.uint8)
    u[inside & (model == C.MODEL_2D)] = C.USER_TO_3D
    u[~inside & (model == C.MODEL_3D)] = C.USER_TO_2D
    return u


def _f32(state):
    return {k: (np.array(v, dtype=F32) if k in KEYS_F else np.array(v, dtype=np.uint8))
            for k, v in state.items()}


def step(s: dict, dt: float, kappa: float) -> tuple[dict, dict]:
    n = len(s["model"])
    P = s["pos_h"]
    user = user_flags(P, s["model"])
    vol = (s["mass"] / s["rho"]).astype(F32)
    rp, col = O.neighbours(P)
    cl = O.classify(P, s["model"], s["ptype"], s["normal"], vol, s["h3d"], user, rp, col)
    flag = O.smooth(s["model"], cl["preflag"], s["last"], rp, col)
    s, _, n = O.remap(s, flag, rp, col)
    s = _f32(s)
    rp, col = O.neighbours(s["pos_h"])
    union, src, _, _ = O.ghost_zone(s, rp, col)
    union = _f32(union)
    U = union["pos_h"]
    urp, ucol = O.neighbours(U)
    rows = np.arange(n)
    coef, status, _ = O.stencils(U, union["model"], urp, ucol, rows=rows)
    out = O.apply(urp, ucol, coef, union["vp"], rows=rows)
    lap = out[:n, 0, 3].astype(F32)
    s["vp"][:, 0] = s["vp"][:, 0] + F32(dt * kappa) * lap
    s["pos_h"][:, 0] = s["pos_h"][:, 0] + F32(dt)
    order = C.cell_order(s["pos_h"])
    s = {k: np.ascontiguousarray(v[order]) for k, v in s.items()}
    return s, {"n": n, "n_all": len(union["model"]), "flag": flag, "near": cl["near"]}


def exact_temperature(xy: np.ndarray, t: float, kappa: float, nr: int = 64,
                      nt: int = 256) -> np.ndarray:
    """T(x, t) of the plane heat equation (diffusivity kappa) from the
    indicator of the disc ADV_DISC moved to (x0 + t, y0): the disc convolved
    with the heat kernel exp(-r^2 / (4 kappa t)) / (4 pi kappa t), by
    Gauss-Legendre quadrature in the radius and the trapezoid rule in the
    angle.  kappa = 0 gives the transported indicator."""
    x0, y0, R = C.ADV_DISC
    cx, cy = x0 + t, y0
    if kappa == 0.0:
        return (((xy[:, 0] - cx) ** 2 + (xy[:, 1] - cy) ** 2) <= R * R).astype(np.float64)
    g, w = np.polynomial.legendre.leggauss(nr)
    rho = 0.5 * R * (g + 1.0)
    wr = 0.5 * R * w
    th = np.linspace(0.0, 2.0 * np.pi, nt, endpoint=False)
    px = cx + rho[:, None] * np.cos(th)[None, :]
    py = cy + rho[:, None] * np.sin(th)[None, :]
    wq = (wr * rho)[:, None] * (2.0 * np.pi / nt)
    out = np.empty(xy.shape[0])
    a = 4.0 * kappa * t
    for s in range(0, xy.shape[0], 2048):
        X = xy[s:s + 2048, 0][:, None, None]
        Y = xy[s:s + 2048, 1][:, None, None]
        r2 = (X - px[None]) ** 2 + (Y - py[None]) ** 2
        out[s:s + 2048] = (np.exp(-r2 / a) * wq[None]).sum((1, 2)) / (np.pi * a)
    return out


def errors(T: np.ndarray, Tref: np.ndarray) -> tuple[float, float]:
    """Relative mean-square and relative maximum errors (Eqs. ep2, epInf)."""
    e2 = float(((T - Tref) ** 2).sum() / (Tref ** 2).sum())
    einf = float(np.abs(T - Tref).max() / np.abs(Tref).max())
    return e2, einf
