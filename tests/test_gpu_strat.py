"""Adaptive stratified sampling (VEGAS+) through the C ABI against the
oracle: FP64 parity on identical samples over consecutive sweeps (estimates,
maps and the integer allocations), FP32 within three standard errors,
bitwise repeatability, and the allocation in the checkpoint state."""
from dataclasses import replace

import numpy as np
import pytest

import workloads as W
from tests._helpers import oracle_sweep, side_integrals, task_arrays
from tests.test_gpu_parity import _compare_fp32

pytestmark = pytest.mark.gpu


def _strat(prob, **kw):
    return replace(prob, processes=tuple(replace(p, strat=1, **kw) for p in prob.processes))


def _f(f0):
    import torch
    return torch.tensor(np.ascontiguousarray(f0), dtype=torch.float64, device="cuda")


def _parity(prob, f0, t=0.0, sweeps=2):
    from paper_2603_28848_gb300 import Collision
    col = Collision(prob, W.PREC_FP64)
    f = _f(f0)
    state = None
    for _ in range(sweeps):
        C, _ = col.eval(f, t)
        Co, _, detail, state = oracle_sweep(prob, f0, t, "f64", state)
    col.check()
    mean, terr = col.task_results()
    om, oe = task_arrays(detail, col.n_tasks)
    keep = np.abs(om) > 0
    assert np.all(np.abs(mean[keep] - om[keep]) <= 1e-5 * np.abs(om[keep]) + 1e-300)
    assert np.all(np.abs(terr[keep] - oe[keep]) <= 1e-4 * np.abs(oe[keep]) + 1e-300)
    n_strat = 0
    for tid, alloc in state.strata.items():
        M, H, m = col.strata(tid)
        assert H == len(alloc) and m is not None
        assert np.array_equal(m, alloc), tid
        n_strat += H > 1
    assert n_strat > 0                   # the problem really stratifies
    maps = col.maps()
    for tid, edges in state.maps.items():
        if abs(om[tid]) == 0:
            continue
        D, nb1 = edges.shape
        assert np.max(np.abs(maps[tid][: D * nb1].reshape(D, nb1) - edges)) < 1e-4, tid
    col.close()


def test_strat_maxwell_fp64_two_sweeps():
    prob, f0 = W.c1_maxwell_2to2(n=8, neval=4000, nitn=2)
    _parity(_strat(prob), f0)


def test_strat_2to3_both_sides_fp64():
    prob, f0 = W.c3_cannibal_2to3(n=6, neval=4000, nitn=2, with_2to2=True)
    _parity(_strat(prob), f0, sweeps=1)


def test_strat_multi_species_expansion_uneven_fp64():
    prob, f0 = W.c4_multi_species(n=6, nmin=1000, nmax=5000, nitn=2)
    _parity(_strat(prob, strat_max_hcubes=512), f0, t=2.0)


def test_strat_fp32_within_three_sigma():
    prob, f0 = W.c3_cannibal_2to3(n=8, neval=8000, nitn=2)
    _compare_fp32(_strat(prob), f0)


def test_strat_is_bitwise_repeatable():
    from paper_2603_28848_gb300 import Collision
    prob, f0 = W.c1_maxwell_2to2(n=8, neval=8000, nitn=3)
    prob = _strat(prob)
    out = []
    for _ in range(2):
        col = Collision(prob, W.PREC_FP32)
        C, err = col.eval(_f(f0), 0.0)
        C2, err2 = col.eval(_f(f0), 0.0)
        out.append((C2.cpu().numpy(), err2.cpu().numpy(), col.strata(3)[2]))
        col.close()
    for a, b in zip(out[0], out[1]):
        assert np.array_equal(a, b)


def test_strat_allocation_is_checkpointed():
    from paper_2603_28848_gb300 import Collision
    prob, f0 = W.c1_maxwell_2to2(n=8, neval=8000, nitn=1)
    col = Collision(_strat(prob), W.PREC_FP64)
    f = _f(f0)
    col.eval(f, 0.0)
    blob = col.save_state()
    m1 = col.strata(5)[2].copy()
    C_a, _ = col.eval(f, 0.0)
    assert not np.array_equal(col.strata(5)[2], m1)
    col.load_state(blob)
    assert np.array_equal(col.strata(5)[2], m1)
    C_b, _ = col.eval(f, 0.0)
    assert np.array_equal(C_a.cpu().numpy(), C_b.cpu().numpy())
    col.close()


def test_strat_task_shapes_follow_the_rule():
    from oracle import stratified as ost
    from paper_2603_28848_gb300 import Collision
    prob, f0 = W.c5_2to4(n=4, neval=20000, nitn=1)
    prob = _strat(prob, strat_max_hcubes=1000)
    col = Collision(prob, W.PREC_FP32)
    for tid in range(col.n_tasks):
        M, H, m = col.strata(tid)
        assert (M, H) == ost.shape(20000, 12, 1000)[:2]
        assert m.sum() == 2500 and m.min() >= 1
    assert col.sweep_samples(0) == col.n_tasks * 20000
    col.close()
