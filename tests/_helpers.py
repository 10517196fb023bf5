"""Shared helpers of the GPU parity tests: run the CUDA path and the oracle
on the same problem and compare task by task."""
import numpy as np

from oracle import collision as ocol
from oracle import tasks as otasks


def oracle_sweep(problem, f, t, mode, state=None, points=None):
    st = state if state is not None else ocol.State()
    C, err, detail = ocol.collision(problem, f, t, st, mode, points=points)
    return C, err, detail, st


def task_arrays(detail, n_tasks):
    mean = np.full(n_tasks, np.nan)
    err = np.full(n_tasks, np.nan)
    for k, (m, e) in detail.items():
        mean[k] = m
        err[k] = e
    return mean, err


def rel_diff(a, b, floor=1e-300):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    scale = np.maximum(np.abs(b), floor)
    d = np.abs(a - b) / scale
    d[(a == 0) & (b == 0)] = 0.0
    return d


def side_integrals(problem):
    return otasks.side_integrals(problem)
