"""Assignment of independent solves to ranks (one process per GPU).

Solves never exchange data, so a multi-GPU run is a partition of the solve
list: no collective touches the data path. The partition is deterministic
(every rank computes the same one from the same list) and balances the
predicted work, cells x steps, with the longest-processing-time rule.
"""
from __future__ import annotations

import os
from typing import List, Sequence


def rank_env():
    """(rank, world_size, local_rank) from the torchrun environment."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def shard_by_cost(costs: Sequence[float], world: int) -> List[List[int]]:
    """Indices of `costs` for each of `world` ranks: largest first, each to the
    currently least-loaded rank (ties to the lowest rank)."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(costs)), key=lambda i: (-float(costs[i]), i))
    load = [0.0] * world
    out: List[List[int]] = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda q: (load[q], q))
        out[r].append(i)
        load[r] += float(costs[i])
    for lst in out:
        lst.sort()
    return out


def shard_workloads(workloads, world: int, rank: int):
    """The workloads rank `rank` owns out of `world`."""
    costs = [w.cells * w.steps for w in workloads]
    return [workloads[i] for i in shard_by_cost(costs, world)[rank]]
