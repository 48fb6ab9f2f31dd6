"""Time loop over the tray shape: every step runs the operator pipeline on the
current cloud, decides model transitions and remaps (Sec. 6: detection, then
the data mapping of Sec. 5), then moves the particles.

    step k:  user criterion (a sphere sweeping the plate)
             neighbours -> classify_pca (flags, film frames)
             stencils -> apply                     (derivatives for the solver)
             remap_switched                        (particle count changes here)
             advect by the smooth displacement field of clouds.tray_velocity
             re-sort into cell order (mafp_cell_order)

The library calls do the path; this module only marshals buffers and applies
the workload's own rules (user criterion, advection) with elementwise torch
operations in a fixed order.  The particle count after each remap is read on
the host once per step, since the next step's launch sizes depend on it.
"""
from __future__ import annotations

import numpy as np
import torch

from . import clouds as Cl
from . import mafp as M
from .pipeline import Pipeline

STATE_KEYS = M.STATE_F4 + M.STATE_F1 + M.STATE_U8


def displacement(xyz: torch.Tensor, vel: dict) -> torch.Tensor:
    """d(x) of clouds.tray_velocity for float32 positions [n, 3]; every
    operation is one rounded float32 op, taken in the documented order."""
    out = torch.zeros_like(xyz)
    for m in range(4):
        kx, ky, kz = (float(v) for v in vel["kappa"][m])
        t = xyz[:, 0] * kx
        t = t + xyz[:, 1] * ky
        t = t + xyz[:, 2] * kz
        t = t + float(vel["phi"][m])
        u = t * float(vel["inv_2pi"])
        u = u - torch.floor(u)
        v = 1.0 - u
        b = u * u
        b = b * v
        b = b * v
        b = b * 16.0
        b = b - float(vel["mean"])
        s = b * float(vel["amp"][m])
        for c in range(3):
            out[:, c] = out[:, c] + s * float(vel["e"][m][c])
    return out


def advect(pos_h: torch.Tensor, model: torch.Tensor, ptype: torch.Tensor, vel: dict):
    """Move particles in place: film and 3D wall particles tangentially (they
    stay on the plate), other 3D particles in full, kept at z >= 0.5 dx."""
    d = displacement(pos_h[:, :3], vel)
    planar = (model == M.MODEL_2D) | (ptype == M.TYPE_WALL)
    d[:, 2] = torch.where(planar, torch.zeros_like(d[:, 2]), d[:, 2])
    pos_h[:, 0] = pos_h[:, 0] + d[:, 0]
    pos_h[:, 1] = pos_h[:, 1] + d[:, 1]
    z = pos_h[:, 2] + d[:, 2]
    pos_h[:, 2] = torch.where(planar, pos_h[:, 2], torch.clamp_min(z, float(vel["zmin"])))


def user_flags(pos_h: torch.Tensor, model: torch.Tensor, step: int) -> torch.Tensor:
    """The sweeping-sphere user criterion of clouds.tray_sphere."""
    c, r, shell = Cl.tray_sphere(step)
    dx = pos_h[:, 0] - float(c[0])
    dy = pos_h[:, 1] - float(c[1])
    dz = pos_h[:, 2] - float(c[2])
    d2 = dx * dx + dy * dy
    d2 = d2 + dz * dz
    inside = d2 < float(r * r)
    trail = (~inside) & (d2 < float((r + shell) ** 2)) & (pos_h[:, 0] < float(c[0]))
    u = torch.zeros_like(model)
    u = torch.where(inside & (model == M.MODEL_2D), torch.full_like(u, M.USER_TO_3D), u)
    u = torch.where(trail & (model == M.MODEL_3D), torch.full_like(u, M.USER_TO_2D), u)
    return u


def state_from_cloud(cloud, cap: int, device="cuda") -> dict:
    s = {}
    for k in STATE_KEYS:
        src = getattr(cloud, "ptype" if k == "type" else k)
        t = torch.zeros((cap,) + src.shape[1:], dtype=torch.float32 if src.dtype == np.float32
                        else torch.uint8, device=device)
        t[: cloud.n] = torch.from_numpy(np.ascontiguousarray(src)).to(device)
        s[k] = t
    return s


class TrayLoop:
    """Device state (two buffers of `cap` rows) and the per-step call sequence."""

    def __init__(self, ctx: M.Context, cloud, cap: int, cap_nnz: int, device="cuda"):
        self.ctx, self.cap, self.dx = ctx, cap, cloud.dx
        self.n = cloud.n
        self.vel = Cl.tray_velocity(cloud.dx)
        self.cur = state_from_cloud(cloud, cap, device)
        self.nxt = {k: torch.zeros_like(v) for k, v in self.cur.items()}
        self.pipe = Pipeline(ctx, cap, cap_nnz, M.F32_REFINED, device)
        self.vol = torch.zeros(cap, dtype=torch.float32, device=device)
        self.user = torch.zeros(cap, dtype=torch.uint8, device=device)
        self.old2new = torch.zeros(cap, dtype=torch.int32, device=device)
        self.n_out = torch.zeros(1, dtype=torch.int64, device=device)
        self.order = torch.zeros(cap, dtype=torch.int32, device=device)

    def cloud_dict(self) -> dict:
        n, S = self.n, self.cur
        self.vol[:n] = S["mass"][:n] / S["rho"][:n]
        return {"pos_h": S["pos_h"][:n], "model": S["model"][:n], "ptype": S["type"][:n],
                "normal": S["normal"][:n], "vol": self.vol[:n], "h3d": S["h3d"][:n],
                "user": self.user[:n], "last": S["last"][:n], "fields": S["vp"][:n]}

    def step(self, k: int) -> dict:
        n, S = self.n, self.cur
        d = self.cloud_dict()
        self.user[:n] = user_flags(S["pos_h"][:n], S["model"][:n], k)
        p = self.pipe
        p.neighbours(d)
        p.classify(d)          # flags, and the film frames the 2D stencils use
        p.stencils(d)
        p.apply(d)
        M.remap_switched(self.ctx, n, S, p.flag[:n], p.row_ptr[: n + 1], p.col, self.nxt,
                         self.cap, self.old2new[:n], self.n_out)
        flag = p.flag[:n]
        counts = torch.stack([(flag == 1).sum(), (flag == 2).sum(),
                              (self.old2new[:n] < 0).sum(), self.n_out[0]]).cpu().numpy()
        to2d, to3d, deleted, n_new = (int(v) for v in counts)
        T = self.nxt
        advect(T["pos_h"][:n_new], T["model"][:n_new], T["type"][:n_new], self.vel)
        # back into cell order (remap appends, advection drifts), so the next
        # neighbour build takes the in-order path
        order = self.order[:n_new]
        M.cell_order(self.ctx, T["pos_h"][:n_new], order)
        idx = order.long()
        for key, v in T.items():
            torch.index_select(v[:n_new], 0, idx, out=S[key][:n_new])
        self.n = n_new
        return {"step": k, "n_in": n, "n_out": n_new, "to2d": to2d, "to3d": to3d,
                "deleted": deleted, "added": n_new - (n - deleted)}

    def mass(self) -> float:
        return float(self.cur["mass"][: self.n].double().sum().item())
