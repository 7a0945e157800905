"""Replica ensembles over several processes (one GPU each).

Independent periodic boxes share nothing during a step, so an ensemble is
split by giving each rank a disjoint set of replicas: no collective in the
data path.  Every replica keeps its stream id (its index in the whole
ensemble), so its trajectory is the same whatever the split.  Only host-side
results are combined: the step time (maximum over ranks) and whatever
per-replica quantities the caller gathers.
"""
from __future__ import annotations

from typing import Dict, List, Sequence

import numpy as np

from . import inputs as I


def replica_cost(system: I.System) -> np.ndarray:
    """Work per replica and step: solvent particles + surface sites + cells
    (the cell pass touches every cell)."""
    out = np.zeros(system.n_rep)
    for r, rep in enumerate(system.replicas):
        sites = sum(system.shapes[s].n_sites for s in rep.body_shapes)
        out[r] = rep.n_solvent + sites + int(np.prod(rep.L))
    return out


def shard(costs: Sequence[float], world_size: int) -> List[List[int]]:
    """Longest-processing-time-first assignment of replicas to ranks: the
    largest remaining replica goes to the least loaded rank (ties to the lower
    rank; equal costs in index order).  Deterministic, so every rank computes
    the same split.  Each rank's list is in ascending replica order."""
    if world_size < 1:
        raise ValueError("world_size must be >= 1")
    c = np.asarray(costs, dtype=np.float64)
    order = sorted(range(len(c)), key=lambda i: (-c[i], i))
    load = [0.0] * world_size
    parts: List[List[int]] = [[] for _ in range(world_size)]
    for i in order:
        r = min(range(world_size), key=lambda k: (load[k], k))
        parts[r].append(i)
        load[r] += c[i]
    return [sorted(p) for p in parts]


def local_system(system: I.System, world_size: int, rank: int) -> I.System:
    """The replicas of `system` that rank `rank` simulates."""
    return system.subset(shard(replica_cost(system), world_size)[rank])


def aggregate_timing(ms_local: float, units_local: float, group=None) -> Dict[str, float]:
    """Whole-job throughput of one timed region: the slowest rank's time and
    the units all ranks processed (torch.distributed, any backend)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(ms_local), float(units_local)], dtype=torch.float64)
    if dist.is_available() and dist.is_initialized():
        if dist.get_backend(group) == "nccl":
            t = t.cuda()
        mx = t.clone()
        dist.all_reduce(mx, op=dist.ReduceOp.MAX, group=group)
        sm = t.clone()
        dist.all_reduce(sm, op=dist.ReduceOp.SUM, group=group)
        ms, units = float(mx[0]), float(sm[1])
    else:
        ms, units = float(t[0]), float(t[1])
    return {"ms": ms, "units": units, "per_s": units / (ms / 1e3) if ms > 0 else float("nan")}
