"""The allocation-free entry point, best_vegas_iteration_noalloc, called
through the C ABI, against the context path (best_collision_eval).

Callers that cannot allocate device memory -- applications whose device
memory comes only from their own pool allocator, or loops that must not take
an allocation's device-wide synchronisation -- use this entry point; its
scratch lives in a static device array.
One VEGAS iteration of a task from the uniform map must reproduce the
context path's estimate and error for that task (same Philox stream), and
the refinement of its training data must give the context path's refined
map.  Each task is computed by two calls in a row, which must agree
exactly (the shared scratch keeps the previous call's contents).
"""
import ctypes

import numpy as np
import pytest

import workloads as W
from oracle import vegas

pytestmark = pytest.mark.gpu


def _run(prob, f0, precision, tasks, rtol, map_tol):
    import torch

    from paper_2603_28848_gb300 import Collision, _lib, config_from_problem

    f = torch.tensor(np.ascontiguousarray(f0), dtype=torch.float64, device="cuda")
    col = Collision(prob, precision)
    col.eval(f, 0.0)
    mean, err = col.task_results()
    maps = col.maps()
    col.close()

    lib = _lib.load()
    cfg, keep = config_from_problem(prob, precision)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for task in tasks:
        p = prob.processes[0]                       # single-process problems
        n_legs = len(p.species_in) + len(p.species_out)
        D, nb, N = 3 * (n_legs - 2), p.nbins, p.neval
        edges = torch.tensor(vegas.uniform_edges(D, nb), dtype=torch.float64, device="cuda").contiguous()
        outs = []
        for _ in range(2):
            out = torch.full((2 + D * nb,), np.nan, dtype=torch.float64, device="cuda")
            st = lib.best_vegas_iteration_noalloc(ctypes.byref(cfg), task, ctypes.c_void_p(f.data_ptr()), 0.0,
                                                  ctypes.c_void_p(edges.data_ptr()), 0, 0,
                                                  ctypes.c_void_p(out.data_ptr()), stream)
            assert st == 0, lib.best_last_error(None)
            torch.cuda.synchronize()
            outs.append(out.cpu().numpy())
        assert np.array_equal(outs[0], outs[1])
        o = outs[0]
        m = o[0] / N
        e = np.sqrt(max(o[1] / N - m * m, 0.0) / (N - 1))
        assert abs(m - mean[task]) <= rtol * abs(mean[task]) + 1e-300, (task, m, mean[task])
        assert abs(e - err[task]) <= 10 * rtol * abs(err[task]) + 1e-300, (task, e, err[task])
        refined = vegas.refine(vegas.uniform_edges(D, nb), o[2:].reshape(D, nb), p.alpha)
        got = maps[task][: D * (nb + 1)].reshape(D, nb + 1)
        assert np.max(np.abs(refined - got)) < map_tol
    del keep


def test_noalloc_matches_context_path_fp64():
    prob, f0 = W.c1_maxwell_2to2(n=16, neval=5001, nitn=1)
    _run(prob, f0, W.PREC_FP64, [0, 1, 9, 22, 31], rtol=1e-5, map_tol=1e-9)
    prob, f0 = W.c3_cannibal_2to3(n=8, neval=3001, nitn=1)
    _run(prob, f0, W.PREC_FP64, [2, 5, 16, 27], rtol=1e-5, map_tol=1e-9)


def test_noalloc_matches_context_path_fp32():
    prob, f0 = W.c1_maxwell_2to2(n=16, neval=5001, nitn=1)
    _run(prob, f0, W.PREC_FP32, [0, 9, 22], rtol=1e-4, map_tol=1e-3)


def _call(lib, prob, precision, task, f, edges, out):
    import torch

    from paper_2603_28848_gb300 import config_from_problem

    cfg, keep = config_from_problem(prob, precision)
    st = lib.best_vegas_iteration_noalloc(ctypes.byref(cfg), task, ctypes.c_void_p(f.data_ptr()), 0.0,
                                          ctypes.c_void_p(edges.data_ptr()), 0, 0,
                                          ctypes.c_void_p(out.data_ptr()),
                                          ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    del keep
    return st


def test_noalloc_rejects_sizes_beyond_its_limits():
    """Every rejection happens on the host before anything is launched: a
    grid above 512 points, more than 64 increments, a stratified process, an
    s-dependent matrix element, and task ids outside the problem."""
    from dataclasses import replace

    import torch

    from paper_2603_28848_gb300 import _lib

    lib = _lib.load()
    dummy = torch.zeros(16, dtype=torch.float64, device="cuda")
    prob, _ = W.c1_maxwell_2to2(n=600, neval=1000, nitn=1)
    assert _call(lib, prob, W.PREC_FP64, 0, dummy, dummy, dummy) == 1          # BEST_ERR_INVALID
    assert b"512" in lib.best_last_error(None)
    base, _ = W.c1_maxwell_2to2(n=16, neval=1000, nitn=1)
    p0 = base.processes[0]
    cases = [(replace(base, processes=(replace(p0, nbins=65),)), 0, b"64"),
             (replace(base, processes=(replace(p0, strat=1),)), 0, b"stratified"),
             (replace(base, processes=(replace(p0, me_coef=(1.0, 0.1, 0.0, 0.0)),)), 0, b"matrix"),
             (base, -1, b"range"),
             (base, 2 * base.grid.n, b"range")]
    for prob, task, word in cases:
        assert _call(lib, prob, W.PREC_FP64, task, dummy, dummy, dummy) == 1, (task, word)
        assert word in lib.best_last_error(None), lib.best_last_error(None)
    torch.cuda.synchronize()
    assert torch.all(dummy == 0)                     # nothing was written


def test_noalloc_flags_invalid_grid_values_with_nan():
    """A grid value of zero (rejected by the spline build, BEST_ERR_NUMERIC on
    the context path) turns every output into NaN; the next call with valid
    values is clean again (the flag lives in the shared scratch and is reset
    by every call).  Through the binding's wrapper."""
    import torch

    from paper_2603_28848_gb300 import BestError, vegas_iteration_noalloc

    prob, f0 = W.c1_maxwell_2to2(n=16, neval=2001, nitn=1)
    f = torch.tensor(np.ascontiguousarray(f0), dtype=torch.float64, device="cuda").reshape(-1)
    bad = f.clone()
    bad[5] = 0.0
    edges = torch.tensor(vegas.uniform_edges(6, 50), dtype=torch.float64, device="cuda").reshape(-1)
    out = torch.zeros(2 + 6 * 50, dtype=torch.float64, device="cuda")
    vegas_iteration_noalloc(prob, W.PREC_FP64, 3, bad, 0.0, edges, out)
    assert torch.all(torch.isnan(out))
    vegas_iteration_noalloc(prob, W.PREC_FP64, 3, f, 0.0, edges, out)
    assert torch.all(torch.isfinite(out)) and out[0].item() > 0.0
    with pytest.raises(BestError):
        vegas_iteration_noalloc(prob, W.PREC_FP64, 3, f, 0.0, edges, out[:-1])
    with pytest.raises(BestError):
        vegas_iteration_noalloc(prob, W.PREC_FP64, 2 * prob.grid.n, f, 0.0, edges, out)
