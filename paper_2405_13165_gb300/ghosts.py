"""Buffer zone of Sec. 5.3 (Alg. 5) on the device: ghost sources, one ghost per
source, the model transition of the ghost cloud (neighbours + remap of the
ghosts alone), and the union of the regular particles with the ghosts it
produced.  Marshalling only; every stage is a libmafp call.  The particle
counts between stages are read on the host (launch sizes depend on them)."""
from __future__ import annotations

import torch

from . import mafp as M
from .pipeline import Pipeline

STATE_KEYS = M.STATE_F4 + M.STATE_F1 + M.STATE_U8


def empty_state(cap: int, dtype=M.F32_REFINED, device="cuda") -> dict:
    rd = M.real_dtype(dtype)
    s = {}
    for k in M.STATE_F4:
        s[k] = torch.zeros(cap, 4, dtype=rd, device=device)
    for k in M.STATE_F1:
        s[k] = torch.zeros(cap, dtype=rd, device=device)
    for k in M.STATE_U8:
        s[k] = torch.zeros(cap, dtype=torch.uint8, device=device)
    return s


class GhostZone:
    """Buffers for ghost clouds of up to cap_ghost intermediate and
    cap_ghost_out transitioned ghosts."""

    def __init__(self, ctx: M.Context, cap_all: int, cap_ghost: int, cap_ghost_out: int,
                 cap_nnz_ghost: int, dtype=M.F32_REFINED, device="cuda"):
        self.ctx, self.dtype = ctx, dtype
        self.cap_all, self.cap_ghost, self.cap_ghost_out = cap_all, cap_ghost, cap_ghost_out
        self.src = torch.zeros(cap_all, dtype=torch.uint8, device=device)
        self.ghost = empty_state(cap_ghost, dtype, device)
        self.flag = torch.zeros(cap_ghost, dtype=torch.uint8, device=device)
        self.ghost_src = torch.zeros(cap_ghost, dtype=torch.int32, device=device)
        self.out = empty_state(cap_ghost_out, dtype, device)
        self.old2new = torch.zeros(cap_ghost, dtype=torch.int32, device=device)
        self.counts = torch.zeros(3, dtype=torch.int64, device=device)
        self.gpipe = Pipeline(ctx, cap_ghost, cap_nnz_ghost, dtype, device)

    def build(self, state: dict, n: int, row_ptr, col) -> tuple[int, int, int]:
        """Append the buffer zone of the n regular particles in `state` (capacity
        cap_all, with their neighbour lists) behind them; returns (n_all,
        intermediate ghosts, transitioned ghosts)."""
        ctx, dt = self.ctx, self.dtype
        M.ghost_sources(ctx, state["model"][:n], row_ptr[: n + 1], col, self.src[:n])
        M.ghost_seed(ctx, n, state, self.src, self.ghost, self.cap_ghost, self.flag,
                     self.ghost_src, self.counts[0:1], dt)
        ng = int(self.counts[0].item())
        if ng > self.cap_ghost:
            raise M.MafpError(M.ECAPACITY, f"{ng} ghosts exceed cap_ghost {self.cap_ghost}")
        ngo = 0
        if ng:
            self.gpipe.neighbours({"pos_h": self.ghost["pos_h"][:ng]})
            M.remap_switched(ctx, ng, self.ghost, self.flag[:ng], self.gpipe.row_ptr[: ng + 1],
                             self.gpipe.col, self.out, self.cap_ghost_out, self.old2new[:ng],
                             self.counts[1:2], dt)
            ngo = int(self.counts[1].item())
            if ngo > self.cap_ghost_out:
                raise M.MafpError(M.ECAPACITY, f"{ngo} ghosts exceed cap_ghost_out")
        M.ghost_append(ctx, n, ngo, self.out, state, self.cap_all, self.counts[2:3], dt)
        n_all = int(self.counts[2].item()) if ngo else n
        if n_all > self.cap_all:
            raise M.MafpError(M.ECAPACITY, f"{n_all} particles exceed cap_all {self.cap_all}")
        return n_all, ng, ngo
