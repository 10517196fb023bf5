"""Variance-driven sample budgets: uneven per-task budgets set by the VEGAS
variance of the previous sweep.

Test infrastructure (see ``oracle/__init__``).

The paper keeps one integrator per grid point and process and reuses it from
step to step (Sec. 3D, App. C), so each integrator's variance is known
before the next evaluation; where the rate is hard to estimate it needs more
evaluations than elsewhere.  Reading (the paper fixes neval per process and
does not spell out a rule for uneven budgets): within a process whose
budgets are variance-driven,

  * task t (a side integral x grid point x gain/loss) that used N_t samples
    per iteration and returned the estimate I_t with MC error e_t has the
    relative variance per sample v_t = N_t (e_t / I_t)^2; a task with
    I_t = 0, or with a value that is not finite, has v_t = 0;
  * the next sweep gives it N_t' = clip(lambda v_t, n_min, n_max), which
    equalises the relative errors (e_t / I_t)^2 = v_t / N_t' = 1 / lambda of
    all tasks that the clip leaves alone, with lambda chosen so that the
    budgets add up to the process's fixed total (the sum of its configured
    budgets): 200 bisection steps on [0, 2 n_max / min_{v_t > 0} v_t], each
    comparing sum_t clip(lambda v_t, n_min, n_max) with the total and keeping
    the lower end, whose sum does not exceed the total;
  * the budget given is lambda v_t rounded down to a multiple of QUANTUM
    samples, then held within [n_min, n_max].

The quantum makes the integer budgets insensitive to the last bits of
lambda v_t, so that two implementations of the rule whose estimates differ
by rounding agree on every budget except where lambda v_t falls within that
rounding of a multiple of the quantum.
"""
import numpy as np

QUANTUM = 256
BISECTIONS = 200


def per_sample_variance(N, mean, err):
    """v_t = N_t (e_t / I_t)^2, 0 where I_t = 0 or a value is not finite."""
    N = np.asarray(N, dtype=np.float64)
    mean = np.asarray(mean, dtype=np.float64)
    err = np.asarray(err, dtype=np.float64)
    v = np.zeros_like(mean)
    ok = (mean != 0.0) & np.isfinite(mean) & np.isfinite(err)
    v[ok] = N[ok] * (err[ok] / mean[ok]) ** 2
    v[~np.isfinite(v)] = 0.0
    return v


def allocate(v, total, n_min, n_max, quantum=QUANTUM):
    """Integer budgets for relative variances v with the fixed total."""
    v = np.asarray(v, dtype=np.float64)
    clip = lambda lam: np.clip(lam * v, n_min, n_max)
    pos = v[v > 0.0]
    lam = 0.0
    if pos.size:
        lo, hi = 0.0, 2.0 * n_max / np.min(pos)
        for _ in range(BISECTIONS):
            mid = 0.5 * (lo + hi)
            if float(np.sum(clip(mid))) < total:
                lo = mid
            else:
                hi = mid
        lam = lo
    N = quantum * np.floor(np.minimum(lam * v, 2.0 * n_max) / quantum)
    return np.clip(N, n_min, n_max).astype(np.int64)


def next_budgets(N, mean, err, total, n_min, n_max):
    """The budgets of the next sweep from the last sweep's budgets, estimates
    and errors of a process's tasks (all arrays in task order)."""
    return allocate(per_sample_variance(N, mean, err), total, n_min, n_max)
