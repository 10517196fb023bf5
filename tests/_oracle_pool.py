"""Runs the oracle's whole-grid collision term over several host processes.

The oracle evaluates tasks one after another; the conservation pins need
every grid point at budgets that take a minute on one core.  The grid points
are dealt out to ``spawn`` worker processes, each of which runs the same
sequence of sweeps on its own points (its own ``State``, so every task sees
the same map history and evaluation counter as in one serial run), and the
per-point results are added up: ``collision(points=...)`` leaves C at the
other points zero.
"""
import multiprocessing as mp
import os

import numpy as np


def _worker(args):
    problems, f, t, points = args
    from oracle import collision as col
    st = col.State()
    out = None
    for prob in problems:
        out = col.collision(prob, f, t, st, "f64", points=points)
    C, err, detail = out
    return C, err * err, detail


def collision_sweeps(problems, f, t=0.0, workers=None):
    """C, its MC error and the per-task detail of the last of the sweeps
    ``problems`` (one Problem per sweep, same grid and processes, budgets
    free), maps carried from sweep to sweep."""
    n = problems[0].grid.n
    workers = workers or max(1, min(8, os.cpu_count() or 1))
    chunks = [list(range(k, n, workers)) for k in range(workers)]
    chunks = [c for c in chunks if c]
    ctx = mp.get_context("spawn")
    with ctx.Pool(len(chunks)) as pool:
        res = pool.map(_worker, [(problems, np.asarray(f), t, c) for c in chunks])
    C = sum(r[0] for r in res)
    var = sum(r[1] for r in res)
    detail = {}
    for r in res:
        detail.update(r[2])
    return C, np.sqrt(var), detail
