"""Autotuner of the launch shapes: the neighbour search's cell tile (cell edge
in percent of max h) and the lanes per particle / per row of classify_pca,
build_stencils, apply_ops and the stencil adjoint.

For a cloud already on the device it times every supported group size of a
stage with CUDA events (a few repetitions, best taken), keeps the fastest,
and caches the choice per population mix (3D fraction and mean row length,
both bucketed) in a JSON file so later runs on similar clouds skip the sweep.
Every shape computes the same results up to summation order.
"""
from __future__ import annotations

import json
import os

import torch

from . import mafp as M

CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build", "tuning.json")
CHOICES = {"stencil3d_group": (8, 16, 32), "stencil2d_group": (4, 8, 16),
           "apply_group": (4, 8, 16), "grad3d_group": (2, 4, 8, 16, 32),
           "grad2d_group": (1, 2, 4, 8, 16), "cell_edge_pct": (100, 115, 130),
           "classify_group": (1, 2, 4, 8, 16)}


def mix_key(d, pipe, n: int) -> str:
    frac3 = float((d["model"][:n] == 0).float().mean().item()) if n else 0.0
    row = float(pipe.row_ptr[n].item()) / max(n, 1)
    return f"f3={round(frac3, 1):.1f}/row={int(round(row / 16.0)) * 16}"


def _time(fn, reps: int = 3) -> float:
    best = float("inf")
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        fn()
        e1.record()
        torch.cuda.synchronize()
        best = min(best, e0.elapsed_time(e1))
    return best


def tune(ctx: M.Context, pipe, d, use_cache: bool = True, verbose: bool = False) -> dict:
    """Pick group sizes for this cloud; returns the chosen tuning and timings."""
    n = d["pos_h"].shape[0]
    pipe.neighbours(d)
    pipe.classify(d)
    torch.cuda.synchronize()
    key = mix_key(d, pipe, n)
    cache = {}
    if use_cache and os.path.exists(CACHE):
        try:
            cache = json.load(open(CACHE))
        except (OSError, ValueError):
            cache = {}
    if use_cache and key in cache:
        ctx.set_tuning(**cache[key]["tuning"])
        return cache[key]
    timings = {}
    best = dict(ctx.tuning())
    # cell tile of the neighbour search (the lists are the same for every edge)
    res = {}
    for pct in CHOICES["cell_edge_pct"]:
        ctx.set_tuning(**{**best, "cell_edge_pct": pct})
        res[pct] = _time(lambda: pipe.neighbours(d))
    best["cell_edge_pct"] = min(res, key=res.get)
    timings["cell_edge_pct"] = res
    ctx.set_tuning(**best)
    pipe.neighbours(d)
    res = {}
    for g in CHOICES["classify_group"]:
        ctx.set_tuning(**{**best, "classify_group": g})
        res[g] = _time(lambda: pipe.classify(d))
    best["classify_group"] = min(res, key=res.get)
    timings["classify_group"] = res
    ctx.set_tuning(**best)
    pipe.classify(d)
    for knob in ("stencil3d_group", "stencil2d_group"):
        res = {}
        for g in CHOICES[knob]:
            ctx.set_tuning(**{**best, knob: g})
            res[g] = _time(lambda: pipe.stencils(d))
        best[knob] = min(res, key=res.get)
        timings[knob] = res
    ctx.set_tuning(**best)
    pipe.stencils(d)
    res = {}
    for g in CHOICES["apply_group"]:
        ctx.set_tuning(**{**best, "apply_group": g})
        res[g] = _time(lambda: pipe.apply(d))
    best["apply_group"] = min(res, key=res.get)
    timings["apply_group"] = res
    ctx.set_tuning(**best)
    # the position adjoint, with the applied operators as its output gradient
    pipe.apply(d)
    gout = pipe.out[:n].clone()
    gpos = torch.empty_like(d["pos_h"])
    for knob in ("grad3d_group", "grad2d_group"):
        res = {}
        for g in CHOICES[knob]:
            ctx.set_tuning(**{**best, knob: g})
            res[g] = _time(lambda: M.build_stencils_backward(
                ctx, d["pos_h"], d["model"], pipe.frame[:n], pipe.row_ptr[: n + 1], pipe.col,
                d["fields"], gout, gpos, pipe.dtype))
        best[knob] = min(res, key=res.get)
        timings[knob] = res
    ctx.set_tuning(**best)
    entry = {"tuning": best, "timings_ms": {k: {str(g): round(v, 4) for g, v in r.items()}
                                            for k, r in timings.items()}, "key": key}
    if verbose:
        print("autotune", entry)
    if use_cache:
        os.makedirs(os.path.dirname(CACHE), exist_ok=True)
        cache[key] = entry
        with open(CACHE, "w") as f:
            json.dump(cache, f, indent=1)
    return entry
