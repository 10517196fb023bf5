"""Host logic of multi-process runs (one process per GPU, torchrun).

The collision integral partitions by grid points (independent tasks, the
paper's MPI design of Sec. 3D).  A sharded evolution gives each rank the
tasks of a contiguous, budget-balanced block of grid points (`shard`, a
context built with points=(lo, hi)); every C evaluation is followed by one
exchange, a sum of the ranks' disjoint C slices (`sharded_step`), after which
every rank applies the same step to its copy of the whole distribution.
bench.py times that design under torchrun (`timed_sharded_steps`: one
workload split over the ranks, strong scaling); independent replicas per
rank are its opt-in alternative.
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


def all_reduce_sum(t):
    """In-place sum over the default process group (no-op without one)."""
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return t


def sharded_step(col, logf, t_dev, dt_dev, dt_request, method="heun", reduce=all_reduce_sum, buffers=None):
    """One Euler or Heun step of a sharded run on this rank.

    ``col`` evaluates C on this rank's grid points (zero elsewhere);
    ``reduce`` sums a tensor over the ranks in place; every rank holds the
    same ``logf`` (whole grid), ``t_dev`` and ``dt_dev`` (device scalars) and
    updates them identically.  ``buffers`` (k1, k2, fstar) may be passed to
    avoid allocations.  Returns the step used."""
    import torch
    k1, k2, fstar = buffers if buffers is not None else (torch.empty_like(logf), torch.empty_like(logf),
                                                           torch.empty_like(logf))
    heun = method == "heun"
    dt_dev.fill_(dt_request)
    col.eval_log(logf, float(t_dev.item()), C=k1)
    reduce(k1)
    col.step_stage(1 if heun else 0, 0, logf, k1, t_dev, dt_dev, fstar=fstar if heun else None)
    dt = float(dt_dev.item())
    if heun:
        col.eval(fstar, float(t_dev.item()) + dt, C=k2)
        reduce(k2)
        col.step_stage(1, 1, logf, k1, t_dev, dt_dev, k2=k2, fstar=fstar)
    return dt


def timed_sharded_steps(col, logf, t_dev, dt_dev, dt_request, method, steps, warmup, clock, barrier=None,
                        reduce=all_reduce_sum):
    """`warmup` untimed, then `steps` timed sharded steps on this rank.

    ``clock()`` returns a time in ms after waiting for the device (the bench
    passes a synchronising CUDA-event clock); ``barrier()`` lines the ranks up
    on both sides of the timed region.  Returns (elapsed ms on this rank,
    whole-grid sweeps done: every rank takes part in each of them)."""
    buffers = None
    try:
        import torch
        buffers = (torch.empty_like(logf), torch.empty_like(logf), torch.empty_like(logf))
    except ImportError:
        pass
    for _ in range(warmup):
        sharded_step(col, logf, t_dev, dt_dev, dt_request, method, reduce=reduce, buffers=buffers)
    if barrier is not None:
        barrier()
    t0 = clock()
    for _ in range(steps):
        sharded_step(col, logf, t_dev, dt_dev, dt_request, method, reduce=reduce, buffers=buffers)
    t1 = clock()
    if barrier is not None:
        barrier()
    return t1 - t0, steps * (2 if method == "heun" else 1)
