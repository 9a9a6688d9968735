"""Instance-parallel batches across ranks (one process per GPU).

A batch of independent problems (uneven grids, each its own medium and load) shards
by instance: each rank owns a subset of the instances, steps them with grouped launches
(``wfft.batch_step``) on its own GPU, and nothing crosses ranks on the data path.  The
only collective gathers the per-instance records (iterations, residuals, timings) on
every rank after the steps, for reporting.

``partition`` balances the ranks by an estimate of the work per instance: the voxel count
times log2 of it (the FFT passes' cost per Krylov iteration), longest first onto the
least-loaded rank; equal loads go to the lower rank, so every rank computes the same
partition without communicating.
"""
from __future__ import annotations

import math
from typing import Dict, List, Sequence


def instance_cost(n) -> float:
    """Work estimate of one instance of grid n = (N1, N2, N3) per Krylov iteration."""
    v = 1
    for x in n:
        v *= int(x)
    return float(v) * math.log2(max(2, v))


def partition(costs: Sequence[float], world: int) -> List[List[int]]:
    """Instance indices per rank (each list ascending); every index appears exactly once."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(costs)), key=lambda i: (-float(costs[i]), i))
    load = [0.0] * world
    out: List[List[int]] = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda k: (load[k], k))
        out[r].append(i)
        load[r] += float(costs[i])
    return [sorted(x) for x in out]


def gather_records(local: Dict[int, dict], world: int) -> Dict[int, dict]:
    """Per-instance records of all ranks ({instance index: record}), on every rank.  A rank
    that owns no instance contributes an empty dict.  Needs an initialised process group
    when world > 1."""
    if world <= 1:
        return dict(local)
    import torch.distributed as dist
    parts: list = [None] * world
    dist.all_gather_object(parts, dict(local))
    out: Dict[int, dict] = {}
    for p in parts:
        for k, v in p.items():
            if k in out:
                raise RuntimeError(f"instance {k} was stepped by two ranks")
            out[k] = v
    return out
