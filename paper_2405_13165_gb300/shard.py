"""Sharding of a batch of independent clouds over ranks (one GPU each).

The clouds share nothing, so a rank takes whole clouds and no collective touches
the data path; only the timing is reduced over ranks.  Clouds go out longest
first, each to the rank with the least assigned cost so far (ties to the lower
rank), which keeps the largest load within one cloud's cost of the mean.  Every
rank computes the same assignment from the same costs, with no communication."""
from __future__ import annotations

import numpy as np


def assign_clouds(costs, world: int) -> list[list[int]]:
    """Indices of the clouds each rank takes, ascending within a rank."""
    if world < 1:
        raise ValueError("world must be >= 1")
    costs = np.asarray(costs, dtype=np.float64)
    order = sorted(range(len(costs)), key=lambda b: (-costs[b], b))
    load = [0.0] * world
    out: list[list[int]] = [[] for _ in range(world)]
    for b in order:
        r = min(range(world), key=lambda k: (load[k], k))
        out[r].append(b)
        load[r] += float(costs[b])
    return [sorted(o) for o in out]


def rank_loads(costs, parts: list[list[int]]) -> list[float]:
    costs = np.asarray(costs, dtype=np.float64)
    return [float(costs[p].sum()) for p in parts]
