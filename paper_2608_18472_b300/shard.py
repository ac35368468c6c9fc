"""Sharding a batch of independent runs over ranks (one GPU per rank) and gathering their observables.

The runs of a batch (a scan of geometries x laser intensities x phases) are independent: a step of one
run never reads another run's state, so a batch splits across GPUs with no exchange in the time loop.
The split balances the work by the longest-processing-time rule on the cost of a run (coefficients x
steps): runs in order of decreasing cost, each to the rank with the least work so far (ties to the
lower rank). After propagation the per-run observables (and final states) are gathered on the host,
once, in the batch's global run order.

Host logic only (no CUDA); the collective is torch.distributed's object gather, so it works with the
gloo backend on CPU and with NCCL between GPU ranks.
"""
from __future__ import annotations

import heapq
from typing import Dict, List, Optional, Sequence


def lpt_partition(costs: Sequence[float], nranks: int) -> List[List[int]]:
    """Runs of each rank (global run indices, ascending) by longest processing time first."""
    if nranks < 1:
        raise ValueError("nranks must be >= 1")
    order = sorted(range(len(costs)), key=lambda i: (-float(costs[i]), i))
    heap = [(0.0, r) for r in range(nranks)]
    shards: List[List[int]] = [[] for _ in range(nranks)]
    for i in order:
        load, r = heapq.heappop(heap)
        shards[r].append(i)
        heapq.heappush(heap, (load + float(costs[i]), r))
    return [sorted(s) for s in shards]


def shard_loads(costs: Sequence[float], shards: Sequence[Sequence[int]]) -> List[float]:
    return [float(sum(costs[i] for i in s)) for s in shards]


def gather_runs(local: Dict[int, object], nruns: int, dst: int = 0, group=None) -> Optional[List[object]]:
    """Gather {global run index: value} from every rank; on `dst` returns the values in global run order
    (every run exactly once), elsewhere None. Single process (torch.distributed not initialised): the
    local values in order."""
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        parts = [local]
        rank = dst
    else:
        rank = dist.get_rank(group)
        world = dist.get_world_size(group)
        parts = [None] * world if rank == dst else None
        dist.gather_object(local, parts, dst=dst, group=group)
    if rank != dst:
        return None
    merged: Dict[int, object] = {}
    for part in parts:
        for k, v in part.items():
            if k in merged:
                raise RuntimeError(f"run {k} reported by two ranks")
            merged[k] = v
    missing = [k for k in range(nruns) if k not in merged]
    if missing:
        raise RuntimeError(f"runs {missing[:8]} missing from the gather")
    return [merged[k] for k in range(nruns)]
