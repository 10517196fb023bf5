"""Multi-process host logic with world_size 2 on CPU (gloo)."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2603_28848_gb300 import dist as bdist


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms, units = bdist.aggregate(10.0 + 5.0 * rank, 2.0 * (rank + 1))
    out[rank] = (ms, units)
    dist.barrier()
    dist.destroy_process_group()


def test_aggregate_two_ranks():
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        port = _free_port()
        procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(timeout=120)
            assert p.exitcode == 0
        assert out[0] == (15.0, 6.0) and out[1] == (15.0, 6.0)


def test_aggregate_without_group_is_local():
    assert bdist.aggregate(3.0, 7.0) == (3.0, 7.0)


@pytest.mark.parametrize("world", [1, 2, 3, 8])
def test_shard_covers_and_balances(world):
    budgets = [int(1e5 * 100 ** (i / 511)) for i in range(512)]
    ranges = [bdist.shard(budgets, r, world) for r in range(world)]
    assert ranges[0][0] == 0 and ranges[-1][1] == 512
    for (a, b), (c, d) in zip(ranges[:-1], ranges[1:]):
        assert b == c
    loads = [sum(budgets[a:b]) for a, b in ranges]
    assert max(loads) <= sum(budgets) / world + max(budgets)


class _Relaxation:
    """Stand-in for a shard's collision context on CPU: C_i = -k_i (f_i - g_i)
    on the shard's grid points, zero elsewhere, and the step stages of
    best_step_stage restated in torch.  Only the orchestration of
    dist.sharded_step (evaluate, exchange, identical stages) is under test."""

    def __init__(self, n, lo, hi, eps=0.3):
        import torch
        self.k = torch.linspace(0.5, 3.0, n, dtype=torch.float64)
        self.g = torch.linspace(0.2, 1.0, n, dtype=torch.float64)
        self.lo, self.hi, self.eps = lo, hi, eps

    def _C(self, f, t, C):
        C.zero_()
        sl = slice(self.lo, self.hi)
        C[sl] = -self.k[sl] * (f[sl] - self.g[sl]) * (1.0 + 0.1 * t)
        return C, None

    def eval_log(self, logf, t, C):
        return self._C(logf.exp(), t, C)

    def eval(self, f, t, C):
        return self._C(f, t, C)

    def step_stage(self, method, stage, logf, k1, t_dev, dt_dev, k2=None, fstar=None):
        if stage == 0:
            f = logf.exp()
            mx = float((k1 / f).abs().max())
            dt = min(float(dt_dev), self.eps / mx) if mx > 0 else float(dt_dev)
            if method == 1:
                fstar.copy_((logf + dt * k1 / f).exp())
            else:
                logf.add_(dt * k1 / f)
                t_dev.add_(dt)
            dt_dev.fill_(dt)
        else:
            logf.add_(0.5 * float(dt_dev) * (k1 / logf.exp() + k2 / fstar))
            t_dev.add_(float(dt_dev))


def _shard_worker(rank, world, port, out, method):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    n = 12
    lo, hi = bdist.shard([1.0] * n, rank, world)
    col = _Relaxation(n, lo, hi)
    logf = torch.linspace(-2.0, 0.5, n, dtype=torch.float64)
    t = torch.tensor([0.0], dtype=torch.float64)
    dt = torch.tensor([0.0], dtype=torch.float64)
    for _ in range(4):
        bdist.sharded_step(col, logf, t, dt, 0.2, method)
    out[rank] = (logf.tolist(), float(t))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("method", ["heun", "euler"])
def test_sharded_steps_on_two_ranks_equal_one_rank(method):
    import torch
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        port = _free_port()
        procs = [ctx.Process(target=_shard_worker, args=(r, 2, port, out, method)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(timeout=120)
            assert p.exitcode == 0
        got = [out[0], out[1]]
    n = 12
    col = _Relaxation(n, 0, n)
    logf = torch.linspace(-2.0, 0.5, n, dtype=torch.float64)
    t = torch.tensor([0.0], dtype=torch.float64)
    dt = torch.tensor([0.0], dtype=torch.float64)
    for _ in range(4):
        bdist.sharded_step(col, logf, t, dt, 0.2, method, reduce=lambda x: x)
    for lf, tt in got:
        assert np.allclose(lf, logf.tolist(), rtol=0, atol=1e-14)
        assert tt == pytest.approx(float(t), rel=1e-15)
    assert float(t) > 0.2            # the steps moved time (some were limited by Eq. (16))


def _timed_worker(rank, world, port, out):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    n = 12
    lo, hi = bdist.shard([1.0] * n, rank, world)
    col = _Relaxation(n, lo, hi)
    logf = torch.linspace(-2.0, 0.5, n, dtype=torch.float64)
    t = torch.tensor([0.0], dtype=torch.float64)
    dt = torch.tensor([0.0], dtype=torch.float64)
    import time
    ms, sweeps = bdist.timed_sharded_steps(col, logf, t, dt, 0.2, "heun", 3, 1, lambda: time.perf_counter() * 1e3,
                                           dist.barrier)
    out[rank] = (logf.tolist(), float(t), sweeps, ms)
    dist.destroy_process_group()


def test_bench_sharded_mode_on_two_ranks_equals_one_rank():
    """The timed loop bench.py runs under torchrun (grid-point shards, one C
    exchange per evaluation): 1 warm-up + 3 timed Heun steps on two gloo ranks
    end where one rank with the whole grid ends, and count 6 whole-grid sweeps."""
    import torch
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        port = _free_port()
        procs = [ctx.Process(target=_timed_worker, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(timeout=120)
            assert p.exitcode == 0
        got = [out[0], out[1]]
    n = 12
    col = _Relaxation(n, 0, n)
    logf = torch.linspace(-2.0, 0.5, n, dtype=torch.float64)
    t = torch.tensor([0.0], dtype=torch.float64)
    dt = torch.tensor([0.0], dtype=torch.float64)
    import time
    ms, sweeps = bdist.timed_sharded_steps(col, logf, t, dt, 0.2, "heun", 3, 1, lambda: time.perf_counter() * 1e3,
                                           reduce=lambda x: x)
    assert sweeps == 6 and ms >= 0.0
    for lf, tt, sw, msr in got:
        assert np.allclose(lf, logf.tolist(), rtol=0, atol=1e-14)
        assert tt == pytest.approx(float(t), rel=1e-15) and sw == 6 and msr >= 0.0


def test_bench_point_costs_match_the_kernel_cost_model():
    """bench.py balances shards by samples x (D + 6) per grid point over its
    tasks, the cost model of the sample kernel's static partition."""
    import importlib.util
    spec = importlib.util.spec_from_file_location("bench", os.path.join(os.path.dirname(os.path.dirname(
        os.path.abspath(__file__))), "bench.py"))
    bench = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(bench)
    import workloads as W
    prob, _ = W.c4_multi_species(n=16, nmin=1000, nmax=100_000)
    c = bench.point_costs(prob)
    sched = np.asarray(prob.processes[0].neval_per_point, dtype=np.float64)
    # AB->AB: 2 sides (one per species), D = 6; AA->AAA: 2 sides, D = 9; AAA->BB: 2 sides, D = 9
    assert np.allclose(c, 2 * sched * (2 * 12 + 2 * 15 + 2 * 15))
