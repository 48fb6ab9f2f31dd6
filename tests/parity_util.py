"""Shared helpers of the GPU parity tests: run the CUDA path through the C ABI
and compare with the oracle.

Error measures (derived in the design notes from FP32 arithmetic):
  stencils  -- per row and operator, max_e |a_e - b_e| / max_e |b_e|
  outputs   -- per output column (field, operator), max_i |a_i - b_i| / max_i |b_i|
Storing inputs and coefficients in FP32 perturbs every output by up to
u * sum_j |c_ij| |u_j - u_i| (u = 2^-24), which for the Laplacian reaches
~1e-5 of the column maximum, so the 1e-4 bar is stated normwise; the
componentwise error (floor 1e-3 of the column maximum) is held to P99_BAR at
its 99th percentile.  Clouds with thin 3D layers or outputs that are small
differences of large terms are held to the plain bar with counted, bounded
exceptions (outputs_vs_bar).
"""
import numpy as np
import torch

from paper_2405_13165_gb300 import mafp as M
from paper_2405_13165_gb300.pipeline import Pipeline, cloud_to_device

TOL = {M.F32_REFINED: 1e-4, M.F32_PLAIN: 2e-3, M.F64: 1e-10}


def run_gpu(cloud, dtype, cap_nnz=None, ctx=None, stages=("nbr", "cls", "st", "ap"),
            cloud_offset=None):
    n = cloud.n
    ctx = ctx or M.Context(max(n, 1))
    cap_nnz = cap_nnz or max(400 * n, 16)
    pipe = Pipeline(ctx, max(n, 1), cap_nnz, dtype)
    d = cloud_to_device(cloud, dtype, cloud_offset=cloud_offset)
    ctx.reset_status()
    if "nbr" in stages:
        pipe.neighbours(d, with_order=True)
    if "cls" in stages:
        pipe.classify(d)
    if "st" in stages:
        pipe.stencils(d)
    if "ap" in stages:
        pipe.apply(d)
    torch.cuda.synchronize()
    st = ctx.status()
    nnz = int(pipe.row_ptr[n].item())
    res = dict(status_block=st, row_ptr=pipe.row_ptr[: n + 1].cpu().numpy(),
               col=pipe.col[:nnz].cpu().numpy(), order=pipe.order[:n].cpu().numpy(),
               flag=pipe.flag[:n].cpu().numpy(), preflag=pipe.preflag[:n].cpu().numpy(),
               near=pipe.near[:n].cpu().numpy(), eig=pipe.eig[:n].double().cpu().numpy(),
               frame=pipe.frame[:n].double().cpu().numpy(),
               hfilm=pipe.hfilm[:n].double().cpu().numpy(),
               coef=pipe.coef[:nnz].double().cpu().numpy(),
               status=pipe.status[:n].cpu().numpy(), cond=pipe.cond[:n].cpu().numpy(),
               out=pipe.out[:n].double().cpu().numpy())
    return res, pipe, d, ctx


def stencil_rowwise_error(rp, a, b, rows=None):
    """max over rows of max_e |a-b| / max_e |b| per operator (rows with b == 0 skipped)."""
    rows = range(len(rp) - 1) if rows is None else rows
    worst = np.zeros(4)
    for i in rows:
        s = slice(rp[i], rp[i + 1])
        bb = np.abs(b[s]).max(0) if rp[i + 1] > rp[i] else np.zeros(4)
        d = np.abs(a[s] - b[s]).max(0) if rp[i + 1] > rp[i] else np.zeros(4)
        ok = bb > 0
        worst[ok] = np.maximum(worst[ok], d[ok] / bb[ok])
        worst[~ok] = np.maximum(worst[~ok], d[~ok])
    return worst


def stencil_rowwise_error_vec(rp, a, b):
    """Vectorised form of stencil_rowwise_error over all rows."""
    n = len(rp) - 1
    rows = np.repeat(np.arange(n), np.diff(rp))
    bmax = np.zeros((n, 4))
    dmax = np.zeros((n, 4))
    np.maximum.at(bmax, rows, np.abs(b))
    np.maximum.at(dmax, rows, np.abs(a - b))
    rel = np.where(bmax > 0, dmax / np.where(bmax > 0, bmax, 1), dmax)
    return rel.max(0) if n else np.zeros(4), rel


def column_error(a, b):
    """Normwise error per output column and the componentwise p99 (floor 1e-3)."""
    scale = np.abs(b).reshape(-1, 16).max(0)
    diff = np.abs(a - b).reshape(-1, 16)
    normwise = diff.max(0) / np.where(scale > 0, scale, 1)
    comp = diff / np.maximum(np.abs(b).reshape(-1, 16), 1e-3 * scale)
    return normwise, np.percentile(comp, 99, axis=0) if comp.size else np.zeros(16)


def sensitivity(rp, col, coef, fields, rows=None):
    """Per output element, sum_j |c_ij^op| |u_j - u_i| (FP64 coefficients): the
    size of the terms an applied output is the sum of.  Near-degenerate rows
    (thin 3D layers) and outputs that are small differences of large terms
    (the constant Laplacian of a quadratic field) have terms far larger than
    the output itself."""
    n = len(rp) - 1
    F = np.asarray(fields, np.float64)
    rows_of = np.repeat(np.arange(n), np.diff(rp))
    keep = np.ones(rows_of.size, bool) if rows is None else np.isin(rows_of, rows)
    r, j, c = rows_of[keep], col[keep], np.abs(np.asarray(coef, np.float64)[keep])
    du = np.abs(F[j] - F[r])
    b = np.zeros((n, 4, 4))
    for f in range(4):
        for op in range(4):
            b[:, f, op] = np.bincount(r, c[:, op] * du[:, f], minlength=n)
    return b


# Outputs held to the plain normwise bar, with counted exceptions: a path that
# evaluates the stencils from FP32 positions cannot resolve an output to better
# than about u * (its terms' size), u = 2^-24 (the rounding of q, p(q) and w
# alone moves the coefficients by ~1e-7 of their row), so an output whose
# terms are 10^3 times the column's largest value can miss a 1e-4 bar.  At most
# EXCEPTION_FRACTION of the outputs may miss it, each by no more than
# EXCEPTION_ULPS units of roundoff of its terms.
EXCEPTION_FRACTION = 1e-2
EXCEPTION_ULPS = 64.0
UNIT_ROUNDOFF = {M.F32_REFINED: 2.0 ** -24, M.F32_PLAIN: 2.0 ** -24, M.F64: 2.0 ** -53}


def outputs_vs_bar(a, b, sens, dtype, zero_rel=1e-6, unit=None):
    """The plain normwise bar TOL[dtype] per output column (field, operator),
    with counted exceptions (see EXCEPTION_FRACTION).  A column whose FP64
    values are all zero to rounding (largest value below zero_rel times its
    largest term size, e.g. d/dz of a depth-constant field) has no relative
    error; it is measured against its largest term size instead.  Returns a
    dict; `ok` holds when the exceptions are few enough and each is bounded.
    unit: the relative agreement of the inputs (default: the unit roundoff of
    the path's precision)."""
    tol = TOL[dtype]
    a = np.asarray(a, np.float64).reshape(-1, 16)
    b = np.asarray(b, np.float64).reshape(-1, 16)
    sens = np.asarray(sens, np.float64).reshape(-1, 16)
    scale = np.abs(b).max(0) if b.size else np.zeros(16)
    term = sens.max(0) if sens.size else np.zeros(16)
    zero = scale <= zero_rel * term
    ref = np.where(zero, term, scale)
    err = np.abs(a - b)
    above = err > tol * ref
    allow = EXCEPTION_ULPS * (UNIT_ROUNDOFF[dtype] if unit is None else unit) * sens
    worst = float((err[above] / np.maximum(allow[above], 1e-300)).max()) if above.any() else 0.0
    comp = err / np.maximum(np.abs(b), 1e-3 * scale)
    p99 = np.percentile(comp[:, ~zero], 99, axis=0) if (~zero).any() and b.size else np.zeros(0)
    n_above = int(above.sum())
    return dict(ok=bool(n_above <= EXCEPTION_FRACTION * max(err.size, 1) and worst <= 1.0),
                above=n_above, outputs=int(err.size), worst_exception=worst,
                normwise=(err / np.where(ref > 0, ref, 1)).max(0) if b.size else np.zeros(16),
                zero_columns=np.nonzero(zero)[0].tolist(), p99=p99)


# Bar of the componentwise p99 (floor 1e-3 of the column maximum): near the
# zero crossings of a column the componentwise error of an FP32 path is its
# normwise error times up to 1e3, so the p99 is held to 10x the normwise bar.
P99_BAR = {M.F32_REFINED: 1e-3, M.F32_PLAIN: 2e-2, M.F64: 1e-9}
