#!/usr/bin/env python
"""Benchmark of the per-particle operator pipeline on synthetic clouds.

One step = one pass of the whole path over the cloud, through the C ABI:
build_neighbours -> classify_pca (+ smoothing) -> remap_switched beside
build_stencils (second stream) -> apply_ops -> apply_ops_backward (scatter
form, second stream) beside build_stencils_backward.  Workload: the jet-impingement cloud (vertical 3D
cylinder r = 0.05 m, h = 0.5 m on a plate with a radial one-layer film disc
r = 1 m), dx bisected to 1M particles, h = 3.5 dx, jitter +-0.1 dx, stored in
cell order.  Inputs are resident in HBM when the timed region starts; L2 is
flushed (256 MB write) before every timed step.

Prints one JSON line (rank 0).  --impl reference times the FP64 CPU oracle on
a bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = ("particles/s for neighbour+PCA+stencil build, apply_ops GB/s; "
          "FP32-refined vs FP64 at 1e-4")
UNIT = "particles/s"


def workload_label(n: int) -> str:
    size = "1M" if n == 1_000_000 else f"{n:,}"
    return (f"jet-impingement cloud, {size} particles (cylinder r=0.05 m h=0.5 m + film disc "
            f"r=1 m)")


# Algorithmic work per unit (see the design notes): bytes of the gather-SpMV,
# flops of the stencil build per same-model neighbour and per particle.
APPLY_BYTES_NNZ = {4: 20, 8: 36}
APPLY_BYTES_N = {4: 88, 8: 168}
ST3_FLOP_NBR, ST3_FLOP_PART = 210.0, 1200.0
ST2_FLOP_NBR, ST2_FLOP_PART = 90.0, 1000.0
STG3_FLOP_NBR, STG3_FLOP_PART = 2.5 * ST3_FLOP_NBR, 2.5 * ST3_FLOP_PART  # adjoint ~2.5x forward
NBR_FLOP_TEST = 11.0   # 3 sub, 2 fma + 1 mul (d^2), add + 2 mul (r^2), compare


def candidate_tests(cloud) -> int:
    """Distance tests of the cell-list search: sum over particles of the
    particle count of the 27 cells around their own cell (cells of edge max h)."""
    P = cloud.pos_h.astype(np.float64)
    lo, hi = P[:, :3].min(0), P[:, :3].max(0)
    c = float(P[:, 3].max()) * (1.0 + 1e-6)
    dim = (np.floor((hi - lo) / c) + 1).astype(np.int64)
    cc = np.clip(np.floor((P[:, :3] - lo) * (1.0 / c)).astype(np.int64), 0, dim - 1)
    grid = np.zeros(tuple(dim[::-1] + 2), np.int64)
    np.add.at(grid, (cc[:, 2] + 1, cc[:, 1] + 1, cc[:, 0] + 1), 1)
    s = np.zeros_like(grid)
    for dz in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                s[1:-1, 1:-1, 1:-1] += grid[1 + dz:grid.shape[0] - 1 + dz,
                                            1 + dy:grid.shape[1] - 1 + dy,
                                            1 + dx:grid.shape[2] - 1 + dx]
    return int(s[cc[:, 2] + 1, cc[:, 1] + 1, cc[:, 0] + 1].sum())


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="mafp", choices=["mafp", "reference"])
    ap.add_argument("--n", type=int, default=1_000_000, help="particle count of the jet cloud")
    ap.add_argument("--cpu-sample", type=int, default=0,
                    help="particles of the CPU-oracle sample (0: the whole cloud)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-batched", action="store_true",
                    help="skip the compact record of the 256-cloud batch in the default run")
    ap.add_argument("--workload", default="jet", choices=["jet", "batched", "tray"],
                    help="jet: the 1M jet-on-plate step (default); batched: 256 independent "
                         "cube-on-sheet clouds, forward pass replayed from a CUDA graph; "
                         "tray: the 16M-particle 20-step loop with model transitions")
    ap.add_argument("--tuning", default=None,
                    help="fixed launch shapes 'g3d,g2d,gapply[,ggrad3d[,ggrad2d]]' instead of the "
                         "autotuner (the adjoint's default 2 and 2)")
    return ap.parse_args()


# --------------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200", "-f", self.path],
                stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "", 1).isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "", 1).isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k] == "Active"})
        loaded = [s for s in sm if mx and s > 0.5 * max(mx)] or sm
        return {"sm_mhz": statistics.median(loaded) if loaded else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows),
                "power_w_max": max((float(r[3]) for r in rows
                                    if r[3].replace(".", "", 1).isdigit()), default=None)}


# ------------------------------------------------------------------ CPU oracle
def cpu_oracle_sample(cloud, m: int):
    """The FP64 oracle on the step's stages over the first m particles (cell
    order; m = the whole cloud by default): neighbours, detection, smoothing,
    remap, stencils, apply, apply transpose and the stencil adjoint, all rows,
    OpenMP over particles on every host core.  Returns (seconds, threads,
    description, particles, the oracle's applied outputs)."""
    import oracle
    sub = cloud.take(np.arange(min(m, cloud.n) if m > 0 else cloud.n))
    t0 = time.perf_counter()
    rp, col = oracle.neighbours(sub.pos_h)
    cl = oracle.classify(sub.pos_h, sub.model, sub.ptype, sub.normal, sub.vol, sub.h3d,
                         sub.user, rp, col)
    flag = oracle.smooth(sub.model, cl["preflag"], sub.last, rp, col)
    oracle.remap(oracle.cloud_state(sub), flag, rp, col)
    coef, status, cond = oracle.stencils(sub.pos_h, sub.model, rp, col)
    out = oracle.apply(rp, col, coef, sub.vp)
    oracle.apply_T(rp, col, coef, out)
    oracle.stencil_grad(sub.pos_h, sub.model, rp, col, sub.vp, out)
    dt = time.perf_counter() - t0
    threads = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    desc = (f"first {sub.n} particles (cell order) of the same cloud: oracle neighbours, "
            f"detection, smoothing, remap, stencils, apply, apply transpose and stencil "
            f"adjoint in FP64 on all rows, OpenMP over particles ({threads} threads)")
    return dt, threads, desc, sub.n, out


COLUMNS = [f"{f}.{op}" for f in ("u", "v", "w", "p") for op in ("dx", "dy", "dz", "lap")]


def error_per_output(a, b):
    """Per output (field . operator) error of `a` against the FP64 oracle
    outputs `b`: normwise max |a - b| / max |b| over the particles, and the
    p99 of the componentwise |a - b| / max(|b|, 1e-3 max |b|)."""
    a = np.asarray(a, np.float64).reshape(-1, 16)
    b = np.asarray(b, np.float64).reshape(-1, 16)
    scale = np.abs(b).max(0)
    diff = np.abs(a - b)
    nw = diff.max(0) / np.where(scale > 0, scale, 1.0)
    comp = diff / np.maximum(np.abs(b), 1e-3 * scale)
    p99 = np.percentile(comp, 99, axis=0)
    return {c: {"normwise": float(f"{nw[k]:.3e}"), "p99": float(f"{p99[k]:.3e}")}
            for k, c in enumerate(COLUMNS)}


def oracle_reorder_spread(cloud):
    """How far the FP64 oracle's own outputs move when every row is summed in
    the reverse order (stencils and apply): the rounding floor that any FP64
    evaluation of the same rows shares, per output column (normwise)."""
    import oracle
    rp, col = oracle.neighbours(cloud.pos_h)
    coef, _, _ = oracle.stencils(cloud.pos_h, cloud.model, rp, col)
    out = oracle.apply(rp, col, coef, cloud.vp)
    col_r = col.copy()
    for i in range(cloud.n):
        col_r[rp[i]:rp[i + 1]] = col[rp[i]:rp[i + 1]][::-1]
    coef_r, _, _ = oracle.stencils(cloud.pos_h, cloud.model, rp, col_r)
    out_r = oracle.apply(rp, col_r, coef_r, cloud.vp)
    e = error_per_output(out_r, out)
    return {"per_output": {k: v["normwise"] for k, v in e.items()},
            "max_normwise": max(v["normwise"] for v in e.values()),
            "what": "FP64 oracle with each row's summation order reversed vs the FP64 oracle "
                    "(normwise per output): the FP64 rounding floor of these rows"}


def analytic_consistency(cloud, out):
    """Consistency of the applied operators with the analytic derivatives of
    the sinusoid fields (a discretisation-error figure, not a parity check):
    3D rows against the gradient and Laplacian, film rows (flat plate, normal
    +z) against the in-plane gradient and the in-plane Laplacian.  Per output:
    normwise max |a - e| / max |e| and the median of |a - e| / max(|e|, 1e-3 max|e|)."""
    if not cloud.field_modes:
        return None
    x = cloud.pos_h[:, :3].astype(np.float64)
    film = cloud.model == 1
    e = np.zeros((cloud.n, 4, 4))
    for f, kx, ky, kz, phi in cloud.field_modes:
        arg = x @ np.array([kx, ky, kz]) + phi
        c, sn = np.cos(arg), np.sin(arg)
        e[:, f, 0] += kx * c
        e[:, f, 1] += ky * c
        e[:, f, 2] += np.where(film, 0.0, kz * c)
        e[:, f, 3] -= np.where(film, kx * kx + ky * ky, kx * kx + ky * ky + kz * kz) * sn
    a = np.asarray(out, np.float64).reshape(-1, 16)
    e = e.reshape(-1, 16)
    scale = np.abs(e).max(0)
    diff = np.abs(a - e)
    nw = diff.max(0) / np.where(scale > 0, scale, 1.0)
    med = np.median(diff / np.maximum(np.abs(e), 1e-3 * scale), axis=0)
    return {"per_output": {c: {"normwise": float(f"{nw[k]:.3e}"), "median": float(f"{med[k]:.3e}")}
                           for k, c in enumerate(COLUMNS)},
            "max_normwise": float(f"{nw.max():.3e}"),
            "what": "FP32-refined outputs vs the analytic derivatives of the sinusoid fields "
                    "(3D rows: gradient and Laplacian; film rows: in-plane gradient and "
                    "Laplacian); discretisation error of the order-2 stencils at h = 3.5 dx, "
                    "largest on one-sided boundary rows"}


def gen_cloud(n):
    from paper_2405_13165_gb300 import clouds as C
    if n == 1_000_000:
        c = C.config_jet_1m()
    else:
        c = C.jet_on_plate(None, n_target=n)
    return C.cell_sorted(c)


# ----------------------------------------------------------------- GPU bench
def bench_gpu(args):
    import torch
    import torch.distributed as dist

    from paper_2405_13165_gb300 import mafp as M
    from paper_2405_13165_gb300.pipeline import Pipeline, cloud_to_device

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    cloud = gen_cloud(args.n)
    n = cloud.n
    dtype = M.F32_REFINED
    ctx = M.Context(n)
    d = cloud_to_device(cloud, dtype, dev)
    # size the CSR buffers from one neighbour build
    probe = torch.empty(1, dtype=torch.int32, device=dev)
    rp = torch.empty(n + 1, dtype=torch.int64, device=dev)
    ctx.reset_status()
    M.build_neighbours(ctx, d["pos_h"], rp, probe, None, None, dtype)
    nnz = int(rp[n].item())
    ctx.reset_status()
    cap_nnz = nnz + 1024
    pipe = Pipeline(ctx, n, cap_nnz, dtype, dev)
    gout = torch.empty(n, 4, 4, dtype=torch.float32, device=dev)
    gfields = torch.empty(n, 4, dtype=torch.float32, device=dev)
    gpos = torch.empty(n, 4, dtype=torch.float32, device=dev)
    cap_out = 2 * n
    state_in = {k: d[k] for k in ("pos_h", "vp", "normal", "rho", "eta", "mass", "diam",
                                  "hfilm", "h3d", "model", "last")}
    state_in["type"] = d["ptype"]
    state_out = {k: torch.empty((cap_out,) + tuple(v.shape[1:]), dtype=v.dtype, device=dev)
                 for k, v in state_in.items()}
    old2new = torch.empty(n, dtype=torch.int32, device=dev)
    n_out = torch.empty(1, dtype=torch.int64, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()
    side_stream = torch.cuda.Stream(dev)
    have_bwd = True
    dsrc = d

    def step(ev=None, src=None, serial=False, outputs_free=None):
        # outputs_free: an event the step waits for before it writes its first
        # output (the flags), e.g. the download of the previous step's results
        nonlocal have_bwd
        d = dsrc if src is None else src
        stream = torch.cuda.current_stream()   # the capturing stream inside a graph capture
        side = stream if serial else side_stream
        sin = state_in if src is None else {**{k: src[k] for k in state_in if k != "type"},
                                            "type": src["ptype"]}
        marks = []
        def mark():
            if ev is not None:
                e = torch.cuda.Event(enable_timing=True)
                e.record(stream)
                marks.append(e)
        mark()
        pipe.neighbours(d)
        mark()
        if outputs_free is not None:
            stream.wait_event(outputs_free)
        pipe.classify(d)
        mark()
        # the remap (memory bound) runs on a second stream beside the stencil
        # build (ALU bound); both only read the neighbour lists and flags
        side.wait_stream(stream)
        M.remap_switched(ctx, n, sin, pipe.flag[:n], pipe.row_ptr[: n + 1], pipe.col,
                         state_out, cap_out, old2new, n_out, dtype, stream=side)
        pipe.stencils(d)
        mark()
        pipe.apply(d)
        mark()
        gout.copy_(pipe.out[:n])
        # the field adjoint (L2 atomics) beside the position adjoint (ALU)
        side.wait_stream(stream)
        M.apply_ops_backward(ctx, pipe.row_ptr[: n + 1], pipe.col, None, pipe.coef, gout,
                             gfields, dtype, stream=side)
        if have_bwd:
            try:
                M.build_stencils_backward(ctx, d["pos_h"], d["model"], pipe.frame[:n],
                                          pipe.row_ptr[: n + 1], pipe.col, d["fields"], gout,
                                          gpos, dtype)
            except M.MafpError as e:
                if e.code != M.ENOTIMPL:
                    raise
                have_bwd = False
        stream.wait_stream(side)
        mark()
        return marks

    from paper_2405_13165_gb300 import autotune
    if args.tuning:
        g = [int(v) for v in args.tuning.split(",")]
        ctx.set_tuning(stencil3d_group=g[0], stencil2d_group=g[1], apply_group=g[2],
                       grad3d_group=g[3] if len(g) > 3 else 2,
                       grad2d_group=g[4] if len(g) > 4 else 2)
        tuned = {"tuning": ctx.tuning(), "source": "command line"}
    else:
        tuned = autotune.tune(ctx, pipe, d, use_cache=False)
    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()
    st = ctx.status()
    if st["code"] != 0:
        raise RuntimeError(f"device status after warm-up: {st}")

    # the whole step (both streams) captured once in a CUDA graph and replayed
    gstream = torch.cuda.Stream(dev)
    gstream.wait_stream(stream)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=gstream):
        step()
    stream.wait_stream(gstream)
    for _ in range(2):
        graph.replay()
    torch.cuda.synchronize()

    # ---- timed region
    sampler = ClockSampler(local)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    sampler.start()
    time.sleep(0.3)
    t_wall0 = time.perf_counter()
    per_step = []
    for _ in range(args.steps):
        flush.fill_(1)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        graph.replay()
        e1.record(stream)
        per_step.append((e0, e1))
    torch.cuda.synchronize()
    t_wall = time.perf_counter() - t_wall0
    clocks = sampler.stop()
    per_step = [a.elapsed_time(b) for a, b in per_step]
    # per-stage times from eager steps with events between the stages
    stages = []
    for _ in range(3):
        flush.fill_(1)
        stages.append(step(ev=True))
    torch.cuda.synchronize()
    names = ["build_neighbours", "classify_pca", "build_stencils (remap beside it)",
             "apply_ops", "backward (field adjoint beside it)"]
    stage_ms = {nm: statistics.mean(m[k].elapsed_time(m[k + 1]) for m in stages)
                for k, nm in enumerate(names)}
    eager_ms = statistics.mean(m[0].elapsed_time(m[-1]) for m in stages)
    total_ms = max_over_ranks(sum(per_step), dev, world)
    ms_step = total_ms / args.steps
    value = world * n / (ms_step * 1e-3)
    st = ctx.status()

    # ---- kernel-level timing on one extra step, the two streams serialised so
    # that each kernel is timed on its own (CUDA events on its stream)
    ctx.profile(True)
    step(serial=True)
    torch.cuda.synchronize()
    prof = ctx.profile_read()
    ctx.profile(False)
    launches_per_step = sum(v[0] for v in prof.values())

    # algorithmic work of the candidate dominant kernels
    model = d["model"]
    rows = torch.repeat_interleave(torch.arange(n, device=dev), pipe.row_ptr[1: n + 1] -
                                   pipe.row_ptr[:n])
    col = pipe.col[:nnz].long()
    same = model[rows] == model[col]
    nbr3 = int((same & (model[rows] == 0)).sum().item())
    nbr2 = int((same & (model[rows] == 1)).sum().item())
    n3 = int((model == 0).sum().item())
    n_cand = candidate_tests(cloud)
    n2 = n - n3
    sm_mhz = clocks.get("sm_mhz") or 1920.0
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    fp32_peak = sms * 128 * 2 * sm_mhz * 1e6 / 1e12   # TFLOP/s at the sampled clock
    peaks = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            peaks = json.load(f)
    except OSError:
        pass
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    hbm_src = "of measured" if "hbm_gbs" in peaks else "of fallback"

    def kernel_ms(prefix):
        hit = [(k, v) for k, v in prof.items() if k.startswith(prefix)]
        if not hit:
            return None, 0
        launches = sum(v[0] for _, v in hit)
        return sum(v[1] for _, v in hit) / max(launches, 1), launches

    kernels = {}
    ms, _ = kernel_ms("k_apply<G=")
    if ms:
        b = APPLY_BYTES_NNZ[4] * nnz + APPLY_BYTES_N[4] * n
        kernels["apply_ops"] = {"bound": "hbm", "achieved": b / (ms * 1e-3) / 1e9, "peak": hbm_peak,
                                "unit": "GB/s", "ms": ms, "algorithmic": b,
                                "peak_src": hbm_src}
    ms, _ = kernel_ms("k_stencil<f32,M=10")
    if ms:
        fl = ST3_FLOP_NBR * nbr3 + ST3_FLOP_PART * n3
        kernels["build_stencils_3d"] = {"bound": "alu", "achieved": fl / (ms * 1e-3) / 1e12,
                                        "peak": fp32_peak, "unit": "TFLOP/s", "ms": ms,
                                        "algorithmic": fl, "peak_src": "FP32 FMA issue rate at sampled clock"}
    ms, _ = kernel_ms("k_stencil<f32,M=6")
    if ms:
        fl = ST2_FLOP_NBR * nbr2 + ST2_FLOP_PART * n2
        kernels["build_stencils_2d"] = {"bound": "alu", "achieved": fl / (ms * 1e-3) / 1e12,
                                        "peak": fp32_peak, "unit": "TFLOP/s", "ms": ms,
                                        "algorithmic": fl, "peak_src": "FP32 FMA issue rate at sampled clock"}
    ms, _ = kernel_ms("k_nbr_mask<float>")
    if ms:
        fl = NBR_FLOP_TEST * n_cand
        kernels["nbr_mask"] = {"bound": "alu", "achieved": fl / (ms * 1e-3) / 1e12, "peak": fp32_peak,
                               "unit": "TFLOP/s", "ms": ms, "algorithmic": fl,
                               "candidate_tests": n_cand,
                               "candidates_per_entry": round(n_cand / max(nnz, 1), 3),
                               "peak_src": "FP32 FMA issue rate at sampled clock"}
    ms, _ = kernel_ms("k_stencil_grad<f32,M=10")
    if ms:
        fl = STG3_FLOP_NBR * nbr3 + STG3_FLOP_PART * n3
        kernels["stencil_adjoint_3d"] = {"bound": "alu", "achieved": fl / (ms * 1e-3) / 1e12,
                                         "peak": fp32_peak, "unit": "TFLOP/s", "ms": ms,
                                         "algorithmic": fl,
                                         "peak_src": "FP32 FMA issue rate at sampled clock"}
    # the dominant kernel: the largest share of the step among those with a roofline
    dominant = max(kernels, key=lambda k: kernels[k]["ms"]) if kernels else None
    traffic = {}
    try:
        # DRAM bytes per launch from an ncu capture, valid only while the
        # kernel's sources are unchanged since the capture
        import hashlib
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            for k, v in json.load(f).items():
                h = hashlib.sha256()
                for src in (v["source"], "paper_2405_13165_gb300/csrc/stencil_common.cuh",
                            "paper_2405_13165_gb300/csrc/internal.cuh"):
                    h.update(open(os.path.join(ROOT, src), "rb").read())
                if h.hexdigest()[:16] == v["source_sha"]:
                    traffic[k] = v["bytes_per_launch"]
    except (OSError, ValueError, KeyError):
        traffic = {}
    roof = None
    if dominant:
        k = kernels[dominant]
        roof = {"kernel": dominant, "bound": k["bound"], "achieved": round(k["achieved"], 2),
                "peak": round(k["peak"], 1), "unit": k["unit"],
                "frac": round(k["achieved"] / k["peak"], 4),
                "traffic": traffic.get(dominant), "peak_source": k["peak_src"],
                "launch_ms": round(k["ms"], 4)}

    # ---- FP64 path on the same cloud (the plain FP64 GPU baseline)
    fp64 = None
    if not args.no_fp64:
        d64 = cloud_to_device(cloud, M.F64, dev)
        pipe64 = Pipeline(ctx, n, cap_nnz, M.F64, dev)
        for _ in range(1):
            pipe64.step(d64)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        k64 = max(2, min(args.steps, 3))
        t64 = 0.0
        for _ in range(k64):
            flush.fill_(1)
            e0.record(stream)
            pipe64.neighbours(d64)
            pipe64.classify(d64)
            pipe64.stencils(d64)
            e1.record(stream)
            torch.cuda.synchronize()
            t64 += e0.elapsed_time(e1)
        t64 /= k64
        pipe64.apply(d64)
        out64 = pipe64.out[:n].cpu().numpy()
        t32 = 0.0
        for _ in range(k64):
            flush.fill_(1)
            e0.record(stream)
            pipe.neighbours(d)
            pipe.classify(d)
            pipe.stencils(d)
            e1.record(stream)
            torch.cuda.synchronize()
            t32 += e0.elapsed_time(e1)
        t32 /= k64
        pipe.apply(d)
        out32 = pipe.out[:n].cpu().numpy()
        fp64 = {"analytic": analytic_consistency(cloud, out32),
                "build_ms_fp64": round(t64, 3), "build_ms_fp32_refined": round(t32, 3),
                "repeats": k64, "speedup": round(t64 / t32, 2),
                "build_particles_per_s_fp32_refined": round(n / (t32 * 1e-3), 1),
                "build_particles_per_s_fp64": round(n / (t64 * 1e-3), 1)}
        del pipe64, d64

    # ---- end to end through the public API with host buffers: every step
    # copies the cloud in from pinned host memory, runs the whole step
    # (forward, remap, adjoints) and copies derivatives, flags, the remapped
    # count and both gradients back.  The copies run on their own stream,
    # pipelined with the compute as a caller streaming clouds would run them:
    # step k+1's inputs go up into a second input buffer while step k
    # computes, and step k's results come down while step k+1 builds its
    # neighbour lists (step k+1 writes its first output only after that
    # download).  Timed from the first upload to the last download.
    e2e = None
    if not args.no_e2e:
        keys = [k for k in d if k != "vp"]
        host = {k: d[k].cpu().pin_memory() for k in keys}
        outs = {"out": pipe.out[:n], "flag": pipe.flag[:n], "n_out": n_out,
                "gfields": gfields, "gpos": gpos}
        back = {k: torch.empty(v.shape, dtype=v.dtype).pin_memory() for k, v in outs.items()}
        h2d = sum(v.numel() * v.element_size() for v in host.values())
        d2h = sum(v.numel() * v.element_size() for v in back.values())
        dd = []
        for _ in range(2):
            buf = {k: torch.empty_like(d[k]) for k in keys}
            buf["vp"] = buf["fields"]
            dd.append(buf)
        copy = torch.cuda.Stream(dev)

        def pipelined(steps):
            ev_in = [torch.cuda.Event(), torch.cuda.Event()]
            ev_used = [torch.cuda.Event(), torch.cuda.Event()]
            ev_out = torch.cuda.Event()
            t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            copy.wait_stream(stream)
            t0.record(copy)
            with torch.cuda.stream(copy):
                for k in keys:
                    dd[0][k].copy_(host[k], non_blocking=True)
            ev_in[0].record(copy)
            for it in range(steps):
                b = it % 2
                stream.wait_event(ev_in[b])
                step(src=dd[b], outputs_free=ev_out if it > 0 else None)
                ev_used[b].record(stream)
                if it + 1 < steps:
                    if it > 0:
                        copy.wait_event(ev_used[1 - b])
                    with torch.cuda.stream(copy):
                        for k in keys:
                            dd[1 - b][k].copy_(host[k], non_blocking=True)
                    ev_in[1 - b].record(copy)
                copy.wait_event(ev_used[b])
                with torch.cuda.stream(copy):
                    for k, v in outs.items():
                        back[k].copy_(v, non_blocking=True)
                ev_out.record(copy)
            t1.record(copy)
            torch.cuda.synchronize()
            return t0.elapsed_time(t1)

        pipelined(2)                                   # warm-up
        e2e_ms = max_over_ranks(pipelined(args.steps), dev, world) / args.steps
        # the results that came back are the step's results
        assert torch.equal(back["flag"], pipe.flag[:n].cpu())
        e2e = {"value": round(world * n / (e2e_ms * 1e-3), 1), "unit": UNIT,
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
               "ms_per_step": round(e2e_ms, 3),
               "path": "pinned host -> device copies of the cloud, the whole step (neighbours, "
                       "detection, remap, stencils, apply, both adjoints), device -> pinned host "
                       "of derivatives, flags, remapped count and gradients; copies on their own "
                       "stream, double-buffered inputs, pipelined with the compute; timed from "
                       "the first upload to the last download; L2 not flushed (the step's "
                       "working set, 1.4 GB of coefficients, is far above L2)"}

    # ---- CPU baseline (rank 0, N = 1 only)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        dt, thr, desc, m, o_out = cpu_oracle_sample(cloud, args.cpu_sample)
        cpu = {"value": round(m / dt, 1), "unit": UNIT, "cores": thr, "kind": "oracle",
               "sample": desc, "seconds": round(dt, 2)}
        # the same oracle on one thread, for context, on the cloud's first 20k particles
        import oracle
        oracle.set_threads(1)
        dt1, _, _, m1, _ = cpu_oracle_sample(cloud, 20_000)
        oracle.set_threads(thr)
        cpu["one_thread"] = {"value": round(m1 / dt1, 1), "unit": UNIT, "seconds": round(dt1, 2),
                             "sample": f"first {m1} particles (cell order), the same stages, "
                                       f"1 thread"}
        if fp64 is not None and m == n:
            # error per output of both GPU paths against the FP64 oracle on the whole cloud
            e32, e64 = error_per_output(out32, o_out), error_per_output(out64, o_out)
            try:
                reorder = oracle_reorder_spread(cloud)
            except Exception as exc:   # a reported figure only: never lose the bench line
                reorder = {"error": f"{type(exc).__name__}: {exc}"}
            fp64["err_per_output"] = {
                "fp32_refined": e32, "fp64": e64,
                "fp32_refined_max_normwise": max(v["normwise"] for v in e32.values()),
                "fp32_refined_max_p99": max(v["p99"] for v in e32.values()),
                "fp64_max_normwise": max(v["normwise"] for v in e64.values()),
                "fp64_oracle_reorder_spread": reorder,
                "bar": {"fp32_refined": 1e-4, "fp64": 1e-10},
                "measure": "per field.operator over all particles: normwise max|a-b|/max|b|, "
                           "p99 of |a-b|/max(|b|, 1e-3 max|b|); b = FP64 oracle"}

    # ---- the batched workload (256 independent clouds), compact record
    batched = None
    if rank == 0 and world == 1 and not args.no_batched:
        batched = run_batched(args, dev, 1, 0, compact=True)

    if rank == 0:
        line = {
            "metric": METRIC, "value": round(value, 1), "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": max(args.warmup, 3), "ms_per_step": round(ms_step, 4),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (seeded jet-on-plate cloud)",
            "config": {"workload": workload_label(args.n), "n_particles": n, "nnz": nnz, "n_3d": n3, "n_2d": n2,
                       "dx": round(cloud.dx, 7), "precision": "FP32 refined, FP64 retakes",
                       "step": "neighbours, detection, remap, stencils, apply, apply transpose"
                               + (", stencil adjoint" if have_bwd else ""),
                       "l2": "flushed (256 MB write) before every timed step",
                       "launch": "the step captured once in a CUDA graph (both streams) and "
                                 "replayed; stage_ms and ms_per_step_eager from eager steps",
                       "parallelism": "replicas" if world > 1 else "single GPU"},
            "stage_ms": {k: round(v, 4) for k, v in stage_ms.items()},
            "ms_per_step_eager": round(eager_ms, 4),
            "build_particles_per_s": round(n / ((stage_ms["build_neighbours"] +
                                                 stage_ms["classify_pca"] +
                                                 stage_ms["build_stencils (remap beside it)"])
                                                * 1e-3), 1),
            "apply_ops_gbs": round(kernels.get("apply_ops", {}).get("achieved", 0.0), 1),
            "roofline": roof,
            "kernels": {k: {kk: (round(vv, 4) if isinstance(vv, float) else vv)
                            for kk, vv in v.items()} for k, v in kernels.items()},
            "fp64_vs_fp32": fp64,
            "batched": batched,
            "tuning": tuned,
            "e2e": e2e,
            "cpu_baseline": cpu,
            "clocks": clocks,
            "gpu_launches": int(launches_per_step * args.steps),
            "kernel_profile_top": [{"kernel": k, "launches": v[0], "ms_per_launch": round(v[1] / v[0], 4)}
                                   for k, v in sorted(prof.items(), key=lambda kv: -kv[1][1])[:12]],
            "device_status": {k: st[k] for k in ("code", "n_fp64_stencil", "n_fp64_eigen",
                                                 "n_deficient", "n_near", "cells_identity")},
            "wall_s_timed_region": round(t_wall, 3),
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


def bench_batched(args):
    """The batched workload alone (--workload batched), one JSON line."""
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", "0")))
    torch.cuda.set_device(dev)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    line = run_batched(args, dev, world, rank)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()


def run_batched(args, dev, world, rank, compact=False):
    """256 independent clouds in one batch (about 12M particles): neighbours,
    detection, stencils and apply over the whole batch, one launch per stage,
    the pass captured once in a CUDA graph and replayed.  Timed both eagerly
    and by graph replay, and the same pass eagerly in FP64 (the plain FP64 GPU
    path); L2 flushed before every timed pass.  compact: a short record for
    the default run's line instead of a full line."""
    import torch

    from paper_2405_13165_gb300 import autotune, clouds as C, mafp as M
    from paper_2405_13165_gb300.pipeline import Pipeline, cloud_to_device

    from paper_2405_13165_gb300 import shard

    # whole clouds per rank (no collective on the data path), longest first
    parts = shard.assign_clouds(C.batched_sizes()[0], world)
    cloud, off = C.config_batched(select=parts[rank])
    n, nb = cloud.n, len(off) - 1
    dtype = M.F32_REFINED
    ctx = M.Context(n)
    d = cloud_to_device(cloud, dtype, dev, cloud_offset=off)
    probe = torch.empty(1, dtype=torch.int32, device=dev)
    rp = torch.empty(n + 1, dtype=torch.int64, device=dev)
    ctx.reset_status()
    M.build_neighbours_batched(ctx, d["cloud_offset"], d["pos_h"], rp, probe)
    nnz = int(rp[n].item())
    ctx.reset_status()
    pipe = Pipeline(ctx, n, nnz + 1024, dtype, dev)
    tuned = autotune.tune(ctx, pipe, d, use_cache=False)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    s = torch.cuda.Stream(dev)
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        for _ in range(max(args.warmup, 3)):
            pipe.step(d, stream=s)
    s.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=s):
        pipe.step(d, stream=s)
    launches = 0
    ctx.profile(True)
    with torch.cuda.stream(s):
        pipe.step(d, stream=s)
    s.synchronize()
    prof = ctx.profile_read()
    ctx.profile(False)
    launches = sum(v[0] for v in prof.values())

    def timed(run, steps):
        tot = 0.0
        with torch.cuda.stream(s):
            for _ in range(steps):
                flush.fill_(1)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(s)
                run()
                e1.record(s)
                s.synchronize()
                tot += e0.elapsed_time(e1)
        return tot / steps

    sampler = ClockSampler(dev.index)
    sampler.start()
    time.sleep(0.3)
    ms_eager = max_over_ranks(timed(lambda: pipe.step(d, stream=s), args.steps), dev, world)
    ms_graph = max_over_ranks(timed(graph.replay, args.steps), dev, world)
    clocks = sampler.stop()
    n_all = int(sum_over_ranks(n, dev, world))
    st = ctx.status()
    if st["code"] != 0:
        raise RuntimeError(f"device status after the batched passes: {st}")
    del graph
    # the same batched pass in FP64 throughout (the plain FP64 GPU path)
    del pipe
    d64 = cloud_to_device(cloud, M.F64, dev, cloud_offset=off)
    pipe64 = Pipeline(ctx, n, nnz + 1024, M.F64, dev)
    with torch.cuda.stream(s):
        pipe64.step(d64, stream=s)
    s.synchronize()
    ms_fp64 = max_over_ranks(timed(lambda: pipe64.step(d64, stream=s), 2), dev, world)
    st64 = ctx.status()
    if st64["code"] != 0:
        raise RuntimeError(f"device status after the FP64 batched passes: {st64}")
    del pipe64, d64
    hit = [v for k, v in prof.items() if k.startswith("k_apply<G=")]
    peaks = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            peaks = json.load(f)
    except OSError:
        pass
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    roof = None
    if hit:
        ms = sum(v[1] for v in hit) / sum(v[0] for v in hit)
        b = APPLY_BYTES_NNZ[4] * nnz + APPLY_BYTES_N[4] * n
        ach = b / (ms * 1e-3) / 1e9
        roof = {"kernel": "apply_ops", "bound": "hbm", "achieved": round(ach, 1),
                "peak": hbm_peak, "unit": "GB/s", "frac": round(ach / hbm_peak, 4),
                "traffic": None, "launch_ms": round(ms, 4),
                "peak_source": "of measured" if "hbm_gbs" in peaks else "of fallback"}
    sizes = np.diff(off)
    workload = (f"batch of {nb} independent cube-on-sheet clouds, sizes log-uniform 2k-200k, "
                f"film fraction U[0.1, 0.9], dx = 0.02 m")
    fp64 = {"ms_per_pass_fp64": round(ms_fp64, 3), "speedup_graph_fp32_refined_vs_fp64":
            round(ms_fp64 / ms_graph, 2), "repeats": 2}
    if compact:
        return {"workload": workload, "n_particles": n, "nnz": nnz, "clouds": nb,
                "ms_per_pass_graph": round(ms_graph, 3), "ms_per_pass_eager": round(ms_eager, 3),
                "particles_per_s": round(n / (ms_graph * 1e-3), 1), "fp64": fp64,
                "apply_roofline": roof, "clocks": clocks, "steps": args.steps,
                "pass": "neighbours, detection, stencils, apply over all clouds, one launch per "
                        "stage, CUDA graph replay; L2 flushed before every timed pass"}
    line = {
        "metric": "particles/s for neighbour+PCA+stencil build+apply over a batch of clouds",
        "value": round(n_all / (ms_graph * 1e-3), 1), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": max(args.warmup, 3), "ms_per_step": round(ms_graph, 4),
        "ms_per_step_eager": round(ms_eager, 4), "higher_is_better": True,
        "scaling": "strong" if world > 1 else "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded cube-on-sheet clouds)",
        "config": {"workload": workload,
                   "n_particles": n_all, "n_particles_rank0": n, "nnz_rank0": nnz,
                   "clouds": len(C.batched_sizes()[0]), "clouds_rank0": nb,
                   "smallest": int(sizes.min()),
                   "largest": int(sizes.max()), "n_2d": int((cloud.model == 1).sum()),
                   "step": "batched neighbours, detection, stencils, apply (CUDA graph replay)",
                   "l2": "flushed (256 MB write) before every timed pass",
                   "parallelism": (f"{world} ranks, whole clouds per rank (longest first)"
                                   if world > 1 else "single GPU")},
        "fp64": fp64,
        "roofline": roof, "tuning": tuned, "clocks": clocks,
        "gpu_launches": int(launches * args.steps),
        "kernel_profile_top": [{"kernel": k, "launches": v[0],
                                "ms_per_launch": round(v[1] / v[0], 4)}
                               for k, v in sorted(prof.items(), key=lambda kv: -kv[1][1])[:12]],
        "device_status": {k: st[k] for k in ("code", "n_fp64_stencil", "n_fp64_eigen",
                                             "n_deficient", "n_near", "cells_identity")},
    }
    return line


def bench_tray(args):
    """The tray loop: 16M particles, each step user criterion, neighbours,
    detection, stencils, apply, remap (about 5 % of the particles switch
    model) and advection; --steps loop steps timed after --warmup steps run on
    a copy of the initial state."""
    import torch

    from paper_2405_13165_gb300 import clouds as C, mafp as M, tray

    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", "0")))
    torch.cuda.set_device(dev)
    cloud = C.config_tray()
    n0 = cloud.n
    cap = int(1.35 * n0)
    ctx = M.Context(cap)
    probe = torch.empty(1, dtype=torch.int32, device=dev)
    rp = torch.empty(n0 + 1, dtype=torch.int64, device=dev)
    pos = torch.from_numpy(cloud.pos_h).to(dev)
    ctx.reset_status()
    M.build_neighbours(ctx, pos, rp, probe)
    nnz0 = int(rp[n0].item())
    ctx.reset_status()
    del pos, rp
    loop = tray.TrayLoop(ctx, cloud, cap=cap, cap_nnz=int(1.35 * nnz0))
    ctx.set_tuning(stencil3d_group=8, stencil2d_group=4, apply_group=8)
    init = {k: v.clone() for k, v in loop.cur.items()}
    for k in range(max(args.warmup, 3)):
        loop.step(k)
    loop.cur = {k: v.clone() for k, v in init.items()}
    loop.n = n0
    m0 = loop.mass()
    torch.cuda.synchronize()
    sampler = ClockSampler(dev.index)
    sampler.start()
    time.sleep(0.3)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    stats = []
    e0.record()
    for k in range(args.steps):
        stats.append(loop.step(k))
    e1.record()
    torch.cuda.synchronize()
    clocks = sampler.stop()
    ms = e0.elapsed_time(e1) / args.steps
    st = ctx.status()
    if st["code"] != 0:
        raise RuntimeError(f"device status after the tray loop: {st}")
    done = sum(s["n_in"] for s in stats)
    frac = [(s["to2d"] + s["to3d"] + s["deleted"] + s["added"]) / s["n_in"] for s in stats]
    ctx.profile(True)
    loop.step(args.steps)
    torch.cuda.synchronize()
    prof = ctx.profile_read()
    ctx.profile(False)
    line = {
        "metric": "particles/s through the tray loop (neighbours, detection, stencils, apply, "
                  "remap, advection per step)",
        "value": round(done / (ms * 1e-3 * args.steps), 1), "unit": UNIT, "n_gpus": 1,
        "steps": args.steps, "warmup": max(args.warmup, 3), "ms_per_step": round(ms, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded tray cloud)",
        "config": {"workload": "tray: 2x1 m film sheet, 256 Gaussian puddles, inclined jet "
                               "column; sweeping-sphere user criterion",
                   "n_particles": n0, "dx": round(cloud.dx, 7), "nnz_step0": nnz0,
                   "l2": "working set (GBs) far above L2", "parallelism": "single GPU",
                   "timing": "CUDA events around the whole loop, one host read per step"},
        "switch_fraction_per_step": [round(f, 4) for f in frac],
        "gpu_launches_per_step": int(sum(v[0] for v in prof.values())),
        "kernel_profile_top": [{"kernel": k, "launches": v[0],
                                "ms_per_launch": round(v[1] / v[0], 4)}
                               for k, v in sorted(prof.items(), key=lambda kv: -kv[1][1])[:12]],
        "mass_drift_rel": (loop.mass() - m0) / m0,
        "clocks": clocks,
        "device_status": {k: st[k] for k in ("code", "n_fp64_stencil", "n_fp64_eigen",
                                             "n_deficient", "n_near")},
    }
    print(json.dumps(line), flush=True)


def max_over_ranks(ms: float, device, world: int) -> float:
    """The slowest rank's time (all ranks get it); the job's time for whole-job
    throughput.  world == 1: returned as is."""
    if world <= 1:
        return float(ms)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.barrier()
    return float(t.item())


def sum_over_ranks(v: float, device, world: int) -> float:
    """Sum of a per-rank count over the ranks (all ranks get it)."""
    if world <= 1:
        return float(v)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(v)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def bench_reference(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    cloud = gen_cloud(args.n)
    m = args.cpu_sample
    import oracle
    oracle.build()
    for _ in range(args.warmup):
        cpu_oracle_sample(cloud, m)   # untimed
    times = []
    for _ in range(args.steps):
        dt, thr, desc, mm, _ = cpu_oracle_sample(cloud, m)
        times.append(dt)
    ms = 1e3 * statistics.mean(times)
    value = mm / (ms * 1e-3)
    line = {"impl": "reference", "metric": METRIC, "value": round(value, 1), "unit": UNIT,
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(ms, 2), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded jet-on-plate cloud)",
            "config": {"workload": workload_label(args.n), "n_particles": cloud.n,
                       "sample_particles": mm},
            "timed_region_s": round(sum(times), 2),
            "cpu_baseline": {"value": round(value, 1), "unit": UNIT, "kind": "oracle",
                             "cores": thr, "sample": desc},
            "e2e": {"value": round(value, 1), "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        bench_reference(args)
    elif args.workload == "batched":
        bench_batched(args)
    elif args.workload == "tray":
        bench_tray(args)
    else:
        bench_gpu(args)


if __name__ == "__main__":
    main()
