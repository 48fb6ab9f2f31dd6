"""Advection-diffusion of a depth-constant temperature over a plate with a 3D
band (Eq. AdvDiff, Sec. 7.2): Lagrangian transport at the uniform velocity
(1, 0, 0), diffusion by explicit Euler with the GFDM Laplacian, 3D model in
x in [1, 2] and film elsewhere, buffer zone rebuilt every step.

    step:  user criterion (2D particles in [1, 2] -> 3D, 3D outside -> 2D)
           neighbours -> classify_pca -> remap_switched   (model transition)
           neighbours -> buffer zone (Alg. 5)              (ghosts appended)
           neighbours of the union -> classify (frames) -> stencils -> apply
           T_i += dt kappa Lap_i T  on the regular particles
           x_i += dt (uniform velocity); re-sort into cell order

The temperature is the first field slot.  Library calls do the path; the
loop's own updates (user criterion, Euler step, transport, permutation)
are elementwise torch operations in a fixed order.
"""
from __future__ import annotations

import numpy as np
import torch

from . import mafp as M
from .ghosts import GhostZone, empty_state
from .pipeline import Pipeline

BAND = (1.0, 2.0)
VELOCITY = 1.0


def user_flags(pos_h: torch.Tensor, model: torch.Tensor) -> torch.Tensor:
    x = pos_h[:, 0]
    inside = (x >= BAND[0]) & (x <= BAND[1])
    u = torch.zeros_like(model)
    u = torch.where(inside & (model == M.MODEL_2D), torch.full_like(u, M.USER_TO_3D), u)
    u = torch.where((~inside) & (model == M.MODEL_3D), torch.full_like(u, M.USER_TO_2D), u)
    return u


def time_step(h: float, kappa: float) -> float:
    """dt = min(0.01, 0.04 dx^2 / kappa), dx = h / 3.5 (explicit Euler well
    inside its stability bound for the GFDM Laplacian)."""
    dx = h / 3.5
    return min(0.01, 0.04 * dx * dx / kappa) if kappa > 0 else 0.01


class AdvDiffLoop:
    def __init__(self, ctx: M.Context, cloud, kappa: float, dt: float, cap: int,
                 cap_nnz: int, device="cuda"):
        self.ctx, self.kappa, self.dt, self.cap = ctx, kappa, dt, cap
        self.n = cloud.n
        keymap = {"type": "ptype"}
        self.cur = empty_state(cap, M.F32_REFINED, device)
        for k, v in self.cur.items():
            a = np.asarray(getattr(cloud, keymap.get(k, k)))
            v[: cloud.n] = torch.from_numpy(a).to(device)
        self.nxt = empty_state(cap, M.F32_REFINED, device)
        self.pipe = Pipeline(ctx, cap, cap_nnz, M.F32_REFINED, device)
        self.gz = GhostZone(ctx, cap, cap // 2, cap, cap_nnz // 2, M.F32_REFINED, device)
        self.user = torch.zeros(cap, dtype=torch.uint8, device=device)
        self.vol = torch.zeros(cap, dtype=torch.float32, device=device)
        self.old2new = torch.zeros(cap, dtype=torch.int32, device=device)
        self.n_out = torch.zeros(1, dtype=torch.int64, device=device)
        self.order = torch.zeros(cap, dtype=torch.int32, device=device)
        self.t = 0.0

    def _dict(self, S, n, user=None):
        self.vol[:n] = S["mass"][:n] / S["rho"][:n]
        return {"pos_h": S["pos_h"][:n], "model": S["model"][:n], "ptype": S["type"][:n],
                "normal": S["normal"][:n], "vol": self.vol[:n], "h3d": S["h3d"][:n],
                "user": self.user[:n] if user is None else user, "last": S["last"][:n],
                "fields": S["vp"][:n]}

    def step(self) -> dict:
        ctx, p = self.ctx, self.pipe
        n, S = self.n, self.cur
        # model transition
        self.user[:n] = user_flags(S["pos_h"][:n], S["model"][:n])
        d = self._dict(S, n)
        p.neighbours(d)
        p.classify(d)
        M.remap_switched(ctx, n, S, p.flag[:n], p.row_ptr[: n + 1], p.col, self.nxt, self.cap,
                         self.old2new[:n], self.n_out)
        n = int(self.n_out.item())
        self.cur, self.nxt = self.nxt, self.cur
        S = self.cur
        # buffer zone
        p.neighbours({"pos_h": S["pos_h"][:n]})
        n_all, ng, ngo = self.gz.build(S, n, p.row_ptr[: n + 1], p.col)
        # Laplacian of T at the regular particles over regular + ghost neighbours
        self.user[:n_all] = 0
        du = self._dict(S, n_all)
        p.neighbours(du)
        p.classify(du)
        p.stencils(du)
        p.apply(du)
        lap = p.out[:n, 0, 3]
        T = S["vp"][:n, 0]
        S["vp"][:n, 0] = T + (self.dt * self.kappa) * lap
        # transport, then back into cell order
        S["pos_h"][:n, 0] = S["pos_h"][:n, 0] + self.dt * VELOCITY
        order = self.order[:n]
        M.cell_order(ctx, S["pos_h"][:n], order)
        idx = order.long()
        for key, v in S.items():
            torch.index_select(v[:n], 0, idx, out=self.nxt[key][:n])
        self.cur, self.nxt = self.nxt, self.cur
        self.n = n
        self.t += self.dt
        return {"n": n, "n_all": n_all, "ghosts": n_all - n}

    def temperature(self):
        n = self.n
        return (self.cur["pos_h"][:n].double().cpu().numpy(),
                self.cur["vp"][:n, 0].double().cpu().numpy(),
                self.cur["model"][:n].cpu().numpy())
