"""The N > 1 host path on CPU ranks (gloo, world size 2): the reductions that
make the job's time the slowest rank's and its particle count the sum, the
assignment of a batch's independent clouds to ranks (every rank computes the
same one, no communication), and the reference arm under
torch.distributed.run (rank 0 prints one line, the other rank exits 0 without
work).  The library's path has no collective on the data path; these are the
only cross-rank steps."""
import json
import os
import socket
import subprocess
import sys

import pytest

pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

_RANK_SCRIPT = r"""
import os, sys
sys.path.insert(0, os.environ["BENCH_ROOT"])
import torch, torch.distributed as dist
dist.init_process_group("gloo")
import bench
rank, world = dist.get_rank(), dist.get_world_size()
got = bench.max_over_ranks(10.0 + 5.0 * rank, torch.device("cpu"), world)
tot = bench.sum_over_ranks(100 + rank, torch.device("cpu"), world)
from paper_2405_13165_gb300 import clouds as C, shard
parts = shard.assign_clouds(C.batched_sizes()[0], world)
everyone = [None] * world
dist.all_gather_object(everyone, parts)
same = all(e == parts for e in everyone)
print("RESULT", rank, got, tot, int(same), ",".join(map(str, parts[rank])), flush=True)
dist.destroy_process_group()
"""


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_time_is_the_slowest_ranks():
    port = _free_port()
    procs = []
    for rank in range(2):
        env = dict(os.environ, RANK=str(rank), WORLD_SIZE="2", LOCAL_RANK=str(rank),
                   MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), BENCH_ROOT=ROOT)
        procs.append(subprocess.Popen([sys.executable, "-c", _RANK_SCRIPT], env=env,
                                      stdout=subprocess.PIPE, stderr=subprocess.PIPE,
                                      text=True))
    outs = []
    for p in procs:
        out, err = p.communicate(timeout=180)
        assert p.returncode == 0, err[-2000:]
        outs.append(out)
    got = sorted(tuple(line.split()[1:]) for o in outs for line in o.splitlines()
                 if line.startswith("RESULT"))
    assert [g[:4] for g in got] == [("0", "15.0", "201.0", "1"), ("1", "15.0", "201.0", "1")]
    # the two ranks' clouds: disjoint, together the whole batch
    mine = [set(map(int, g[4].split(","))) for g in got]
    assert not (mine[0] & mine[1]) and mine[0] | mine[1] == set(range(256))


def test_single_rank_time_is_unchanged():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(12.5, None, 1) == 12.5


def test_reference_arm_under_torchrun_prints_one_line():
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), "bench.py",
           "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0",
           "--cpu-sample", "2000"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-3000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, r.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2
    assert d["value"] > 0 and d["cpu_baseline"]["kind"] == "oracle"
    assert d["e2e"]["h2d_bytes_per_step"] == 0


def test_cloud_assignment_balances_whole_clouds():
    sys.path.insert(0, ROOT)
    import numpy as np

    from paper_2405_13165_gb300 import clouds as C, shard
    costs = C.batched_sizes()[0]
    for world in (1, 2, 3, 4, 8):
        parts = shard.assign_clouds(costs, world)
        flat = sorted(b for p in parts for b in p)
        assert flat == list(range(len(costs)))              # each cloud exactly once
        loads = shard.rank_loads(costs, parts)
        # longest-first greedy: no rank exceeds the mean by more than one cloud
        assert max(loads) <= costs.sum() / world + costs.max() + 1e-6
        assert parts == shard.assign_clouds(costs, world)    # deterministic
    assert shard.assign_clouds([5.0, 5.0], 2) == [[0], [1]]
    assert shard.assign_clouds(np.ones(3), 5)[3:] == [[], []]
    with pytest.raises(ValueError):
        shard.assign_clouds([1.0], 0)


def test_rank_share_builds_the_same_clouds():
    sys.path.insert(0, ROOT)
    import numpy as np

    from paper_2405_13165_gb300 import clouds as C
    kw = dict(nclouds=6, n_lo=200, n_hi=1500)
    full, off = C.config_batched(**kw)
    sel = [4, 1]
    part, poff = C.config_batched(select=sel, **kw)
    for k, b in enumerate(sel):
        a = slice(off[b], off[b + 1])
        q = slice(poff[k], poff[k + 1])
        np.testing.assert_array_equal(full.pos_h[a], part.pos_h[q])
        np.testing.assert_array_equal(full.model[a], part.model[q])
