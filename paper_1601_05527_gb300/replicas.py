"""Host-side logic of multi-GPU runs (one process per GPU, no data exchange).

A single graph does not shard without a halo exchange in every sweep, so a
run on N GPUs is N independent replicas of the workload; a batch of graphs
shards by whole graphs.  Nothing here touches the data path: it assigns work
to ranks and combines timings with ``torch.distributed`` (NCCL on GPUs, gloo
in the CPU tests).
"""
from __future__ import annotations

import heapq


def shard_by_size(sizes, world_size: int, rank: int) -> list[int]:
    """Indices of the graphs that ``rank`` runs: longest-processing-time
    greedy on the given sizes (largest graph to the least-loaded rank, ties
    to the lower rank), returned in increasing index order.  Every rank
    computes the same assignment, so no communication is needed."""
    if world_size < 1 or not 0 <= rank < world_size:
        raise ValueError("need 0 <= rank < world_size")
    order = sorted(range(len(sizes)), key=lambda i: (-int(sizes[i]), i))
    heap = [(0, r) for r in range(world_size)]
    mine = []
    for i in order:
        load, r = heapq.heappop(heap)
        if r == rank:
            mine.append(i)
        heapq.heappush(heap, (load + int(sizes[i]), r))
    return sorted(mine)


def max_over_ranks(x: float, device=None) -> float:
    """Largest value of ``x`` over all ranks (the slowest rank's time); ``x``
    itself when no process group is initialised."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x: float, device=None) -> float:
    """Sum of ``x`` over all ranks (units processed by the whole job)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def whole_job_rate(units_this_rank: float, seconds_this_rank: float, device=None) -> float:
    """Throughput of the whole job: units of all ranks over the slowest rank's time."""
    return sum_over_ranks(units_this_rank, device) / max_over_ranks(seconds_this_rank, device)
