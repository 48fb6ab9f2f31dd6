"""The tray loop on the CPU: the FP64 oracle for every stage of a step, the
workload's own rules (sweeping-sphere user criterion, advection by the
displacement field of clouds.tray_velocity) written again here in numpy
float32, operation for operation as the field's definition states.  State
between steps is stored in float32, as the GPU loop stores it."""
import numpy as np

import oracle as O
from paper_2405_13165_gb300 import clouds as C

F32 = np.float32
KEYS_F = ("pos_h", "vp", "normal", "rho", "eta", "mass", "diam", "hfilm", "h3d")
KEYS_U8 = ("model", "ptype", "last")


def displacement(xyz: np.ndarray, vel: dict) -> np.ndarray:
    out = np.zeros_like(xyz)
    for m in range(4):
        kx, ky, kz = vel["kappa"][m]
        t = xyz[:, 0] * kx
        t = t + xyz[:, 1] * ky
        t = t + xyz[:, 2] * kz
        t = t + vel["phi"][m]
        u = t * vel["inv_2pi"]
        u = u - np.floor(u)
        v = F32(1.0) - u
        b = u * u
        b = b * v
        b = b * v
        b = b * F32(16.0)
        b = b - vel["mean"]
        s = b * vel["amp"][m]
        for c in range(3):
            out[:, c] = out[:, c] + s * vel["e"][m][c]
    return out


def advect(state: dict, vel: dict) -> None:
    P = state["pos_h"]
    d = displacement(P[:, :3], vel)
    planar = (state["model"] == C.MODEL_2D) | (state["ptype"] == C.TYPE_WALL)
    d[planar, 2] = F32(0.0)
    P[:, 0] = P[:, 0] + d[:, 0]
    P[:, 1] = P[:, 1] + d[:, 1]
    z = P[:, 2] + d[:, 2]
    P[:, 2] = np.where(planar, P[:, 2], np.maximum(z, vel["zmin"]))


def user_flags(P: np.ndarray, model: np.ndarray, step: int) -> np.ndarray:
    c, r, shell = C.tray_sphere(step)
    dx = P[:, 0] - F32(c[0])
    dy = P[:, 1] - F32(c[1])
    dz = P[:, 2] - F32(c[2])
    d2 = dx * dx + dy * dy
    d2 = d2 + dz * dz
    inside = d2 < F32(r * r)
    trail = (~inside) & (d2 < F32((r + shell) ** 2)) & (P[:, 0] < F32(c[0]))
    u = np.zeros(model.shape, np.uint8)
    u[inside & (model == C.MODEL_2D)] = C.USER_TO_3D
    u[trail & (model == C.MODEL_3D)] = C.USER_TO_2D
    return u


def initial_state(cloud) -> dict:
    s = {k: np.array(getattr(cloud, k), dtype=F32) for k in KEYS_F}
    s.update({k: np.array(getattr(cloud, k), dtype=np.uint8) for k in KEYS_U8})
    return s


def step(state: dict, k: int, vel: dict, rows=None) -> tuple[dict, dict]:
    """One loop step (ending with the re-sort into cell order); returns (next
    state, what the step computed)."""
    P = state["pos_h"]
    model = state["model"]
    rp, col = O.neighbours(P)
    coef, status, _ = O.stencils(P, model, rp, col, rows=rows)
    out = O.apply(rp, col, coef, state["vp"], rows=rows)
    user = user_flags(P, model, k)
    vol = (state["mass"] / state["rho"]).astype(F32)
    cl = O.classify(P, model, state["ptype"], state["normal"], vol, state["h3d"], user, rp, col)
    flag = O.smooth(model, cl["preflag"], state["last"], rp, col)
    nxt, old2new, n_out = O.remap(state, flag, rp, col)
    nxt = {k: (np.array(v, dtype=F32) if k in KEYS_F else np.array(v, dtype=np.uint8))
           for k, v in nxt.items()}
    advect(nxt, vel)
    order = C.cell_order(nxt["pos_h"])
    nxt = {k: np.ascontiguousarray(v[order]) for k, v in nxt.items()}
    info = dict(row_ptr=rp, col=col, coef=coef, status=status, out=out, flag=flag,
                near=cl["near"], preflag=cl["preflag"], old2new=old2new, n_out=n_out,
                user=user)
    return nxt, info
