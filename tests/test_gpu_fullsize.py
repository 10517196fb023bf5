"""Sampled parity at the benchmark's full size: the two-species Bose-Einstein
2 -> 2 workload (128 log points, 512 tasks, 1e6 samples per task) in the
launch configuration bench.py times: the FP32 sample kernel chosen by the
autotuner and the staged chunk partition of a full iteration (6.1e9 cost
units, far above 16 x grid chunks of the minimum chunk size).

One VEGAS iteration from uniform maps, so that the GPU and the oracle see the
same samples (the first iteration of every timed sweep computes exactly
this); twelve tasks spread over both side integrals, the grid and both terms
are recomputed by the oracle one by one (FP64 arithmetic on the FP32-form
uniforms) and must agree to FP32 rounding: largest relative difference below
2e-3 and median below 2e-4 (the one-iteration FP32 bounds of the parity
tests for this workload's rounding, measured at 9.9e-4 / 5.9e-5 on a 24-point
grid)."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

POINTS = (5, 29, 53, 77, 101, 125)


def test_bose_2to2_full_size_sampled_tasks_match_oracle():
    import torch

    from oracle import collision as ocol
    from oracle import vegas
    from oracle.tasks import side_integrals
    from paper_2603_28848_gb300 import Collision
    prob, f0 = W.c2_bose_2to2()
    assert prob.grid.n == 128 and prob.processes[0].neval == 1_000_000
    one = prob.with_budget(nitn=1)
    col = Collision(one, W.PREC_FP32)
    try:
        f = torch.tensor(np.ascontiguousarray(f0), dtype=torch.float64, device="cuda")
        col.autotune(f, 0.0)                 # leaves maps, budgets and counter as they were
        assert col.call_counter == 0
        col.eval(f, 0.0)
        col.check()
        mean, _ = col.task_results()
    finally:
        col.close()
    sis = side_integrals(one)
    dists = ocol.distributions(one, f0, 0.0)
    n = one.grid.n
    rel = []
    for k, i in enumerate(POINTS):
        for si_idx, si in enumerate(sis):
            term = (k + si_idx) % 2
            p = one.processes[si.process]
            om = ocol.evaluate_task(one, si_idx, si, i, term, f0, 0.0, vegas.uniform_edges(si.dim, p.nbins), 0,
                                    "f32", dists)[0]
            g = mean[(si_idx * n + i) * 2 + term]
            assert np.isfinite(g) and om != 0.0, (si_idx, i, term, g, om)
            rel.append(abs(g - om) / abs(om))
    rel = np.array(rel)
    assert len(rel) == 2 * len(POINTS)
    assert rel.max() < 2e-3 and np.median(rel) < 2e-4, rel
