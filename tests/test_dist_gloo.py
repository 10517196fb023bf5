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
