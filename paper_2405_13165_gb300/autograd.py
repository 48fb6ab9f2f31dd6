"""torch.autograd.Function over the stencil build and application.

`gfdm_operators(ctx, pos_h, fields, row_ptr, col, model, frame)` returns the
applied operators out[i, f] = (d_x, d_y, d_z, Lap) of the four fields
(Eq. GFDM_Definition with the stencils of Sec. 2.3).  Its backward runs the
library's hand-written kernels: the exact transpose of apply_ops for the
fields (scattered with atomic adds) and the stencil adjoint (moment matrix and
Cholesky recomputed per particle) for the positions.  Neighbour sets and models
are held fixed.  `frame` must be the tangent frame classify_pca computes from
the same positions: the backward includes its dependence on the positions
(through the PCA normal of each film row), so a caller that moves the particles
recomputes it before the next forward.  The smoothing length column of pos_h
gets no gradient.
"""
from __future__ import annotations

import torch

from . import mafp as M


class _GfdmOperators(torch.autograd.Function):
    @staticmethod
    def forward(fctx, pos_h, fields, mctx, row_ptr, col, model, frame, dtype):
        n = pos_h.shape[0]
        nnz = col.numel()
        rd = M.real_dtype(dtype)
        coef = torch.empty((max(nnz, 1), 4), dtype=rd, device=pos_h.device)
        status = torch.empty(n, dtype=torch.uint8, device=pos_h.device)
        cond = torch.empty(n, dtype=torch.float32, device=pos_h.device)
        out = torch.empty((n, 4, 4), dtype=rd, device=pos_h.device)
        M.build_stencils(mctx, pos_h.detach(), model, frame, row_ptr, col, coef, status, cond,
                         dtype)
        M.apply_ops(mctx, row_ptr, col, coef, fields.detach(), out, dtype)
        fctx.save_for_backward(pos_h, fields, row_ptr, col, model, frame, coef)
        fctx.mctx = mctx
        fctx.dtype = dtype
        return out

    @staticmethod
    def backward(fctx, gout):
        pos_h, fields, row_ptr, col, model, frame, coef = fctx.saved_tensors
        mctx, dtype = fctx.mctx, fctx.dtype
        gout = gout.contiguous()
        n = pos_h.shape[0]
        gpos = gfields = None
        if fctx.needs_input_grad[1]:
            # scatter form of the adjoint: no transpose map for a one-off backward
            gfields = torch.empty_like(fields)
            M.apply_ops_backward(mctx, row_ptr, col, None, coef, gout, gfields, dtype)
        if fctx.needs_input_grad[0]:
            gpos = torch.empty_like(pos_h)
            M.build_stencils_backward(mctx, pos_h.detach(), model, frame, row_ptr, col,
                                      fields.detach(), gout, gpos, dtype)
        return gpos, gfields, None, None, None, None, None, None


def gfdm_operators(mctx: M.Context, pos_h, fields, row_ptr, col, model, frame,
                   dtype: int = M.F32_REFINED):
    """Differentiable applied GFDM operators, shape [n, 4, 4]."""
    return _GfdmOperators.apply(pos_h, fields, mctx, row_ptr, col, model, frame, dtype)
