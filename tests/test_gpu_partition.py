"""The work partition of every VEGAS iteration covers each task's sample
groups exactly once (best_partition_groups): the host-built partition of a
full-size iteration (the staged chunks of decreasing cost), the equal chunks
of a small one, and the partition the device rebuilds after variance-driven
budgets moved, both staged (multi-species workload at its full size) and
equal-chunked (a small case).  A task of N samples in D dimensions has
ceil(N / G) groups, G = 4 / gcd(D, 4) on the FP32 path (four uniforms per
Philox block) and 2 / gcd(D, 2) on the FP64 path."""
from math import gcd

import numpy as np
import pytest

import workloads as W
from tests._helpers import side_integrals

pytestmark = pytest.mark.gpu


def _expected_groups(prob, budgets, f32, iteration):
    n = prob.grid.n
    per = 4 if f32 else 2
    out = np.zeros(len(budgets), dtype=np.int64)
    for k, si in enumerate(side_integrals(prob)):
        G = per // gcd(si.dim, per)
        active = prob.processes[si.process].nitn > iteration
        for i in range(n):
            for term in (0, 1):
                tid = (k * n + i) * 2 + term
                out[tid] = -(-int(budgets[tid]) // G) if active else 0
    return out


def _check_all_iterations(col, prob, f32):
    budgets = col.budgets()
    for it in range(max(p.nitn for p in prob.processes)):
        got = col.partition_groups(it)
        want = _expected_groups(prob, budgets, f32, it)
        assert np.array_equal(got, want), (it, np.flatnonzero(got != want)[:5])


def test_full_size_staged_partition_covers_every_group():
    prob, _ = W.c2_bose_2to2()
    from paper_2603_28848_gb300 import Collision
    col = Collision(prob, W.PREC_FP32)
    try:
        _check_all_iterations(col, prob, True)
        assert col.partition_groups(0).sum() == 512 * 500_000
    finally:
        col.close()


@pytest.mark.parametrize("size", ["full", "small"])
def test_device_rebuilt_partition_after_budget_change(size):
    import torch

    from paper_2603_28848_gb300 import Collision
    if size == "full":
        prob, f0 = W.c4_multi_species(variance_budgets=True)
    else:
        prob, f0 = W.c4_multi_species(n=12, nmin=1000, nmax=4000, nitn=2, variance_budgets=True)
    col = Collision(prob, W.PREC_FP32)
    try:
        before = col.budgets()
        _check_all_iterations(col, prob, True)
        col.eval(torch.tensor(f0, dtype=torch.float64, device="cuda"), 2.0)
        col.check()
        after = col.budgets()
        assert not np.array_equal(before, after)          # the budgets moved ...
        _check_all_iterations(col, prob, True)            # ... and the device's partition follows them
    finally:
        col.close()


def test_fp64_small_partition():
    prob, f0 = W.c3_cannibal_2to3(n=8, neval=2999, nitn=2, with_2to2=True)
    from paper_2603_28848_gb300 import Collision
    col = Collision(prob, W.PREC_FP64)
    try:
        _check_all_iterations(col, prob, False)
    finally:
        col.close()
