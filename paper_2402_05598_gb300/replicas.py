"""Replica bookkeeping for multi-GPU runs. Solves are independent, so N GPUs run N replicas
with disjoint instance sets and no collective on the data path; only the timing frame is
shared: a barrier before and after, the slowest rank's time, and the sum of solved
instances (throughput = all ranks' solves / slowest rank's time)."""
from __future__ import annotations


def rank_seeds(rank: int, per_rank: int, base: int = 10000) -> range:
    """Instance seeds of one rank: disjoint blocks of `per_rank` seeds."""
    return range(base + per_rank * rank, base + per_rank * (rank + 1))


def reduce_timing(total_ms: float, solved: int, device=None):
    """(max over ranks of total_ms, sum over ranks of solved); identity without a process group."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(total_ms), int(solved)
    t = torch.tensor([float(total_ms)], dtype=torch.float64, device=device)
    s = torch.tensor([float(solved)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(s, op=dist.ReduceOp.SUM)
    return float(t.item()), int(round(s.item()))
