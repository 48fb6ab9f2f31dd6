"""Device-resident buffers and the call sequence of one pass of the operator
pipeline: build_neighbours -> classify_pca -> build_stencils -> apply_ops
(-> remap_switched).  Marshalling only; every step is a libmafp call."""
from __future__ import annotations

import numpy as np
import torch

from . import mafp as M

CLOUD_KEYS = ("pos_h", "model", "ptype", "normal", "vp", "rho", "eta", "mass", "diam", "hfilm",
              "h3d", "user", "last")


def cloud_to_device(cloud, dtype=M.F32_REFINED, device="cuda", pin=False, cloud_offset=None):
    """Copy a generated Cloud to device tensors of the call's real type
    (with the batch's int64 cloud offsets when given)."""
    rd = M.real_dtype(dtype)
    out = {}
    for k in CLOUD_KEYS:
        a = getattr(cloud, k)
        t = torch.from_numpy(np.ascontiguousarray(a))
        if t.dtype in (torch.float32, torch.float64):
            t = t.to(rd)
        out[k] = t.to(device, non_blocking=False)
    out["vol"] = torch.from_numpy(np.ascontiguousarray(cloud.vol)).to(rd).to(device)
    out["fields"] = out["vp"]
    if cloud_offset is not None:
        out["cloud_offset"] = torch.as_tensor(np.asarray(cloud_offset, np.int64)).to(device)
    return out


class Pipeline:
    """Pre-allocated outputs for clouds of up to cap_n particles / cap_nnz entries."""

    def __init__(self, ctx: M.Context, cap_n: int, cap_nnz: int, dtype=M.F32_REFINED,
                 device="cuda"):
        self.ctx, self.dtype, self.cap_n, self.cap_nnz = ctx, dtype, cap_n, cap_nnz
        rd = M.real_dtype(dtype)
        z = lambda *s, dt=rd: torch.zeros(*s, dtype=dt, device=device)
        self.row_ptr = z(cap_n + 1, dt=torch.int64)
        self.col = z(cap_nnz, dt=torch.int32)
        self.nnz = z(1, dt=torch.int64)
        self.order = z(cap_n, dt=torch.int32)
        self.flag = z(cap_n, dt=torch.uint8)
        self.preflag = z(cap_n, dt=torch.uint8)
        self.near = z(cap_n, dt=torch.uint8)
        self.eig = z(cap_n, 4)
        self.frame = z(cap_n, 8)
        self.hfilm = z(cap_n)
        self.coef = z(cap_nnz, 4)
        self.status = z(cap_n, dt=torch.uint8)
        self.cond = z(cap_n, dt=torch.float32)
        self.out = z(cap_n, 4, 4)

    def neighbours(self, d, with_order=False, stream=None):
        """Eq. Nbd; a cloud dict holding "cloud_offset" (int64 [B+1], device) is
        a batch of independent clouds and takes the batched build."""
        n = d["pos_h"].shape[0]
        order = self.order[:n] if with_order else None
        if d.get("cloud_offset") is not None:
            M.build_neighbours_batched(self.ctx, d["cloud_offset"], d["pos_h"],
                                       self.row_ptr[: n + 1], self.col, self.nnz, order,
                                       self.dtype, stream)
        else:
            M.build_neighbours(self.ctx, d["pos_h"], self.row_ptr[: n + 1], self.col, self.nnz,
                               order, self.dtype, stream)

    def classify(self, d, stream=None):
        n = d["pos_h"].shape[0]
        M.classify_pca(self.ctx, d["pos_h"], d["model"], d["ptype"], d["normal"], d["vol"],
                       d["h3d"], d["user"], d["last"], self.row_ptr[: n + 1], self.col,
                       self.flag[:n], self.preflag[:n], self.eig[:n], self.frame[:n],
                       self.hfilm[:n], self.near[:n], self.dtype, stream)

    def stencils(self, d, stream=None):
        n = d["pos_h"].shape[0]
        M.build_stencils(self.ctx, d["pos_h"], d["model"], self.frame[:n], self.row_ptr[: n + 1],
                         self.col, self.coef, self.status[:n], self.cond[:n], self.dtype, stream)

    def apply(self, d, fields=None, stream=None):
        n = d["pos_h"].shape[0]
        M.apply_ops(self.ctx, self.row_ptr[: n + 1], self.col, self.coef,
                    d["fields"] if fields is None else fields, self.out[:n], self.dtype, stream)

    def step(self, d, stream=None):
        """One pass of the forward path (no host synchronisation)."""
        self.neighbours(d, stream=stream)
        self.classify(d, stream=stream)
        self.stencils(d, stream=stream)
        self.apply(d, stream=stream)

    def csr(self, n):
        nnz = int(self.row_ptr[n].item())
        return self.row_ptr[: n + 1], self.col[:nnz]


def reorder_cloud(cloud, order: np.ndarray):
    """Permute a Cloud into the library's cell order (what a Lagrangian code
    keeps between steps so later neighbour searches take the sorted path)."""
    return cloud.take(np.asarray(order, dtype=np.int64))


def cell_sorted(cloud, ctx: M.Context | None = None, device="cuda"):
    """Return the cloud permuted into cell order (one neighbour build on the GPU)."""
    own = ctx is None
    ctx = ctx or M.Context(cloud.n)
    d = cloud_to_device(cloud, device=device)
    n = cloud.n
    row_ptr = torch.empty(n + 1, dtype=torch.int64, device=device)
    # only the order is needed; a one-entry col buffer makes the fill pass skip
    col = torch.empty(1, dtype=torch.int32, device=device)
    order = torch.empty(n, dtype=torch.int32, device=device)
    ctx.reset_status()
    M.build_neighbours(ctx, d["pos_h"], row_ptr, col, None, order)
    torch.cuda.synchronize()
    ctx.reset_status()
    if own:
        ctx.close()
    return reorder_cloud(cloud, order.cpu().numpy())
