"""Host logic of multi-process runs (one process per GPU, torchrun).

The collision integral partitions by grid points (independent tasks, the
paper's MPI design of Sec. 3D), so ranks need no data-path collective:
bench.py runs an independent replica of the workload on every rank (weak
scaling) and only reduces its timing.  `shard` is the contiguous,
budget-balanced partition of grid points a sharded evolution would use.
"""
import numpy as np


def aggregate(ms_local, units_local, device=None):
    """(max over ranks of the elapsed ms, sum over ranks of the units).

    Without an initialised process group it returns the local values."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(ms_local), float(units_local)
    t = torch.tensor([float(ms_local)], dtype=torch.float64, device=device)
    u = torch.tensor([float(units_local)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


def shard(budgets, rank, world):
    """Contiguous range [lo, hi) of grid points for `rank`, balancing the
    per-point sample budgets (cumulative cost split into equal parts)."""
    b = np.asarray(budgets, dtype=np.float64)
    cum = np.concatenate([[0.0], np.cumsum(b)])
    total = cum[-1]
    lo = int(np.searchsorted(cum, total * rank / world, side="left"))
    hi = int(np.searchsorted(cum, total * (rank + 1) / world, side="left"))
    if rank == world - 1:
        hi = len(b)
    return min(lo, len(b)), min(hi, len(b))
