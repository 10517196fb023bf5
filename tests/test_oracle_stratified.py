"""Pins of the adaptive stratified sampling (VEGAS+) oracle: the shape and
allocation rules, a hand-computed estimate, an analytic integral, the
reduction to classic VEGAS with one hypercube, and the stratified collision
term against the independent quadrature reduction."""
from dataclasses import replace

import numpy as np
import pytest
from scipy.special import erf

from oracle import collision as col
from oracle import philox, vegas
from oracle import reference as ref
from oracle import stratified as st
from oracle.tasks import side_integrals
from workloads import STAT_MB, Grid, Problem, Process, Species


def test_shape_rule():
    assert st.shape(10 ** 6, 3, 65536) == (31, 29791, 125000)
    assert st.shape(2 * 10 ** 6, 12, 65536) == (2, 4096, 250000)
    assert st.shape(4 * 10 ** 6, 6, 65536) == (6, 46656, 500000)
    assert st.shape(10 ** 6, 3, 4096) == (16, 4096, 125000)
    assert st.shape(16, 3, 65536) == (1, 1, 2)
    for N in (8, 100, 3001, 77777, 10 ** 6):
        for D in (3, 6, 9, 12):
            M, H, J = st.shape(N, D, 65536)
            assert H == M ** D and J == N // 8
            assert M == 1 or 4 * H <= J
            assert 4 * (M + 1) ** D > J or (M + 1) ** D > 65536


def test_allocation_rules():
    J, H = 1000, 64
    u = st.uniform_allocation(J, H)
    assert u.sum() == J and u.min() >= 1 and u.max() - u.min() <= 1 and u[0] >= u[-1]
    s2 = np.ones(H)
    s2[5] = 16.0
    m = st.allocate(s2, J, 0.75)
    assert m.sum() == J and m.min() >= 1
    d = s2 ** 0.375
    base = 1 + np.floor((J - H) * d / d.sum())
    assert np.all(m - base >= 0) and np.all(m - base <= 1)
    rest = J - int(base.sum())
    assert np.array_equal(m - base, (np.arange(H) < rest).astype(int)) and m[5] > 2 * m[6]
    assert np.array_equal(st.allocate(np.zeros(H), J, 0.75), u)


def test_estimate_by_hand():
    # two hypercubes: 1 item (8 samples) and 2 items (16 samples)
    m = np.array([1, 2])
    S1 = np.array([8.0, 48.0])            # means 1 and 3
    S2 = np.array([8.0 + 7.0, 16 * 9.0 + 30.0])
    mean, var, s2 = st.estimate(S1, S2, m)
    assert np.isclose(mean, (1.0 + 3.0) / 2)
    assert np.allclose(s2, [7.0 / 7.0, 30.0 / 15.0])
    assert np.isclose(var, (1.0 / 8 + 2.0 / 16) / 4)


def _strat_integral(fun, D, N, nitn, beta, seed_task):
    """Stratified MC of fun over [0,1]^D with the oracle's rules (identity map)."""
    M, H, J = st.shape(N, D, 65536)
    alloc = st.uniform_allocation(J, H)
    out = []
    for it in range(nitn):
        item_h = np.repeat(np.arange(H), alloc)
        u = philox.uniforms(99, seed_task, it, 0, 8 * J, D, "f64")
        h = item_h[np.arange(8 * J) // 8]
        x = (st.digits(h, M, D) + u) / M
        w = fun(x)
        S1 = np.bincount(h, weights=w, minlength=H)
        S2 = np.bincount(h, weights=w * w, minlength=H)
        mean, var, s2 = st.estimate(S1, S2, alloc)
        out.append((mean, var))
        alloc = st.allocate(s2, J, beta)
    return out, alloc, M


def test_gaussian_peak_integral_and_adaptation():
    """A narrow 3-d Gaussian: every iteration within 3.5 sigma of the erf
    closed form; the adapted allocation puts the most samples at the peak
    and lowers the variance well below the first (uniform) iteration's."""
    c, s = 0.3, 0.05
    fun = lambda x: np.exp(-np.sum((x - c) ** 2, axis=1) / (2 * s * s))
    exact = (s * np.sqrt(np.pi / 2) * (erf((1 - c) / (s * np.sqrt(2))) + erf(c / (s * np.sqrt(2))))) ** 3
    out, alloc, M = _strat_integral(fun, 3, 80_000, 4, 0.75, 5)
    for mean, var in out:
        assert abs(mean - exact) < 3.5 * np.sqrt(var)
    assert out[-1][1] < 0.3 * out[0][1]
    hpeak = int(np.sum((np.floor(c * M).astype(int)) * M ** np.arange(3)))
    assert alloc[hpeak] == alloc.max()


def _mb_problem(strat, max_h=65536, neval=40_000, nitn=3):
    grid = Grid(16, 0.01, 30.0, True)
    proc = Process("pp", (0, 0), (0, 0), 1.0, 0.2, neval, nitn, 0.5, 50, strat=strat, strat_max_hcubes=max_h)
    return Problem(grid, (Species("phi", STAT_MB, 0.0),), (proc,), seed=21)


def test_one_hypercube_reduces_to_classic_vegas():
    """H = 1: the same samples, the same estimate and the same map as the
    classic path (N a multiple of 8)."""
    pc, ps = _mb_problem(0, neval=4000), _mb_problem(1, max_h=1, neval=4000)
    q = col.grid_q(pc.grid)
    f = (0.5 * np.exp(-q / 1.5))[None, :]
    dists = col.distributions(pc, f, 0.0)
    si = side_integrals(pc)[0]
    e0 = vegas.uniform_edges(6, 50)
    a = col.evaluate_task(pc, 0, si, 7, 1, f, 0.0, e0, 0, "f64", dists)
    b = col.evaluate_task(ps, 0, si, 7, 1, f, 0.0, e0, 0, "f64", dists)
    assert b[4] is not None and list(b[4]) == [500]
    for (ma, va), (mb, vb) in zip(a[3], b[3]):
        assert np.isclose(ma, mb, rtol=1e-12) and np.isclose(va, vb, rtol=1e-9)
    assert np.max(np.abs(a[2] - b[2])) < 1e-12


def test_stratified_collision_term_matches_reduction():
    """Stratified MC of the massless MB loss term with the Gaussian of width
    0.2 against the independent centre-of-mass quadrature, within 3.5 sigma."""
    prob = _mb_problem(1)
    q = col.grid_q(prob.grid)
    f = (0.5 * np.exp(-q / 1.5))[None, :]
    dists = col.distributions(prob, f, 0.0)
    si = side_integrals(prob)[0]
    d = dists[0]
    for i in (4, 8):
        mean, err, _, iters, alloc = col.evaluate_task(prob, 0, si, i, 1, f, 0.0, vegas.uniform_edges(6, 50), 0,
                                                       "f64", dists)
        red = ref.two_body_cm_smeared(q[i], (0, 0, 0, 0), f[0, i], d, d, d, (0, 0, 0, 0), 0.2, term="loss",
                                      r_cut=(prob.grid.q_min, prob.grid.q_max), n_omega=24)
        assert abs(mean - red) < 3.5 * err, (i, mean, red, err)
        assert alloc.sum() == 40_000 // 8


def test_sweep_keeps_allocation_in_state():
    prob = _mb_problem(1, neval=8000, nitn=1)           # J = 1000 items, M = 2, H = 64
    prob = replace(prob, grid=Grid(6, 0.05, 20.0, True))
    q = col.grid_q(prob.grid)
    f = (0.5 * np.exp(-q / 1.5))[None, :]
    state = col.State()
    col.collision(prob, f, 0.0, state)
    assert len(state.strata) == 2 * prob.grid.n
    first = {k: v.copy() for k, v in state.strata.items()}
    col.collision(prob, f, 0.0, state)
    assert any(not np.array_equal(first[k], state.strata[k]) for k in first)
    assert all(v.sum() == 1000 and len(v) == 64 for v in state.strata.values())


@pytest.mark.parametrize("N", [8, 9, 15])
def test_budget_rounds_down_to_items(N):
    p = Process("pp", (0, 0), (0, 0), neval=N, strat=1)
    assert col.task_budget(p, 0) == 8
