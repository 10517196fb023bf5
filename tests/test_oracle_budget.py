"""Pins of the variance-driven budget rule (oracle/budget.py): hand-worked
allocations, the clip and water-filling cases, the degenerate inputs, and
the rule's purpose on a Monte Carlo problem (the relative errors of the next
sweep come out more even at the same total)."""
import numpy as np

from oracle import budget as ob
from oracle import collision as col
from oracle.tasks import side_integrals, task_id
from workloads import STAT_MB, Grid, Problem, Process, Species

Q = ob.QUANTUM


def test_proportional_when_no_clip_is_active():
    """v = (1, 2, 3, 4) c and a total of 40000: lambda v = (4000, 8000, 12000,
    16000), rounded down to multiples of 256."""
    N = ob.allocate(np.array([1.0, 2.0, 3.0, 4.0]) * 0.37, 40_000, 1, 10 ** 9)
    assert list(N) == [3840, 7936, 11776, 15872]


def test_clipped_task_leaves_its_share_to_the_others():
    """v = (1, 1, 1, 1000), n_max = 20000, total 50000: the last task is held
    at 20000 and the other three share 30000 equally (10000 -> 9984)."""
    N = ob.allocate(np.array([1.0, 1.0, 1.0, 1000.0]), 50_000, 1000, 20_000)
    assert list(N) == [9984, 9984, 9984, 20000]


def test_floor_clip_and_degenerate_inputs():
    # a task with zero, non-finite or undefined relative variance gets n_min
    v = ob.per_sample_variance([100, 100, 100, 100], [0.0, np.nan, 2.0, 1.0], [1.0, 1.0, 0.2, np.inf])
    assert v[0] == v[1] == v[3] == 0.0 and np.isclose(v[2], 1.0, rtol=1e-15)
    N = ob.allocate(v, 40_000, 2048, 10 ** 6)
    assert N[0] == N[1] == N[3] == 2048 and N[2] == Q * ((40_000 - 3 * 2048) // Q)
    # every v zero: all at n_min; n_min above the share: all at n_min
    assert list(ob.allocate(np.zeros(3), 9000, 1000, 5000)) == [1000] * 3
    assert list(ob.allocate(np.ones(3), 2000, 1000, 5000)) == [1000] * 3
    # total above what the clips allow: every task at n_max
    assert list(ob.allocate(np.array([1.0, 5.0]), 10 ** 7, 1000, 5000)) == [5000, 5000]


def test_random_allocations_respect_total_bounds_and_order():
    rng = np.random.default_rng(7)
    for _ in range(50):
        T = int(rng.integers(2, 60))
        v = rng.lognormal(0.0, 2.0, T) * (rng.random(T) > 0.1)
        n_min, n_max = 1024, 1024 * int(rng.integers(2, 200))
        total = float(rng.uniform(T * n_min, T * n_max))
        N = ob.allocate(v, total, n_min, n_max)
        assert np.all((N >= n_min) & (N <= n_max))
        assert N.sum() <= total + 1e-9
        reach = np.where(v > 0, n_max, n_min).sum()      # the most the clips allow
        assert N.sum() > min(total, reach) - T * Q - 1     # only the rounding is lost ...
        order = np.argsort(v, kind="stable")
        assert np.all(np.diff(N[order]) >= 0)               # ... and larger variance never gets less
        free = (N > n_min) & (N < n_max - Q)
        if np.count_nonzero(free) >= 2:                    # unclipped tasks: N within a quantum of lambda v
            lam = N[free] / v[free]
            assert np.all(np.abs(lam * v[free] - lam.max() * v[free]) <= Q * 1.0001)


def test_sweeps_use_the_budgets_and_even_out_relative_errors():
    """MB 2->2 with a flat configured budget: after the first sweep every
    task's next budget comes from its relative variance; the second sweep
    evaluates each task with exactly that budget (re-running one task alone
    reproduces it), keeps the total, and spreads the relative errors less
    than the same sweep with the flat budget."""
    m = 1.0
    grid = Grid(10, 0.05, 12.0, True)
    base = dict(coupling=1.0, sigma_E=0.1, neval=8192, nitn=2, alpha=0.5, nbins=20)
    prob_v = Problem(grid, (Species("phi", STAT_MB, m),),
                     (Process("pp", (0, 0), (0, 0), budget=1, neval_min=1024, neval_max=65536, **base),), seed=31)
    prob_f = Problem(grid, (Species("phi", STAT_MB, m),), (Process("pp", (0, 0), (0, 0), **base),), seed=31)
    q = col.grid_q(grid)
    f = (0.5 * np.exp(-np.sqrt(q * q + m * m)) + 0.2 * np.exp(-(q - 2.0) ** 2 / 0.5))[None, :]
    sv, sf = col.State(), col.State()
    col.collision(prob_v, f, 0.0, sv)
    col.collision(prob_f, f, 0.0, sf)
    T = 2 * grid.n
    assert sorted(sv.budgets) == list(range(T))
    first = dict(sv.budgets)
    assert sum(first.values()) <= 8192 * T and len(set(first.values())) > 3
    maps_before = {k: v.copy() for k, v in sv.maps.items()}
    _, _, dv = col.collision(prob_v, f, 0.0, sv)
    _, _, df = col.collision(prob_f, f, 0.0, sf)
    # one task re-run alone with its budget and map gives the sweep's result
    si = side_integrals(prob_v)[0]
    tid = task_id(0, 4, 1, grid.n)
    mean, err, *_ = col.evaluate_task(prob_v, 0, si, 4, 1, f, 0.0, maps_before[tid], 1, N=first[tid])
    assert (mean, err) == dv[tid]
    rel = lambda d: np.array([d[k][1] / abs(d[k][0]) for k in range(T)])
    spread = lambda r: np.std(np.log(r))
    assert spread(rel(dv)) < 0.7 * spread(rel(df))
