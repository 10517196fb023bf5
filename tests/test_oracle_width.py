"""Pins of the fractional Gaussian width of App. C and its controller: the
Monte Carlo term against an independent quadrature of the same smeared
definition, the narrow-width limit against the exact-delta closed form, and
the controller's rule (narrow, widen, hold, clamp) on a sweep."""
from dataclasses import replace

import numpy as np
import pytest

from oracle import collision as col
from oracle import reference as ref
from oracle import vegas
from oracle import width as ow
from oracle.tasks import side_integrals
from workloads import (STAT_BE, STAT_MB, WIDTH_ADAPTIVE, WIDTH_FRACTIONAL, Grid, Problem, Process,
                       Species)


def _bose_bump(q, m, T=1.0):
    return 1.0 / np.expm1(np.sqrt(q * q + m * m) / T) + 0.3 * np.exp(-(q - 3.0) ** 2 / (2 * 0.5 ** 2))


@pytest.mark.parametrize("case", ["mb_massless_loss", "be_massive_gain"])
def test_mc_matches_fractional_smeared_reduction(case):
    """Fractional width w = 0.05: the Monte Carlo term equals the quadrature
    of the same definition (omega = E_in - E_out, sigma = w (E_in + E_out)/2)
    within 3.5 sigma (48 nodes in omega / sigma; converged to well below
    the MC error at these momenta)."""
    w = 0.05
    pts = (6, 8, 11)
    if case == "mb_massless_loss":
        m, stat, eta, term = 0.0, STAT_MB, 0.0, 1
        fq = lambda q: 0.5 * np.exp(-q / 1.5)
    else:
        m, stat, eta, term = 0.5, STAT_BE, 1.0, 0
        fq = lambda q: _bose_bump(q, 0.5)
    grid = Grid(16, 0.01, 30.0, True)
    proc = Process("pp", (0, 0), (0, 0), 1.0, 0.2, 40_000, 4, 0.5, 50, width_mode=WIDTH_FRACTIONAL, width=w)
    prob = Problem(grid, (Species("phi", stat, m),), (proc,), seed=13)
    q = col.grid_q(grid)
    f = fq(q)[None, :]
    dists = col.distributions(prob, f, 0.0)
    si = side_integrals(prob)[0]
    for i in pts:
        mean, err, *_ = col.evaluate_task(prob, 0, si, i, term, f, 0.0, vegas.uniform_edges(6, 50), 0, "f64",
                                            dists)
        d = dists[0]
        red = ref.two_body_cm_fractional(q[i], (m, m, m, m), f[0, i], d, d, d, (eta,) * 4, w,
                                         term="gain" if term == 0 else "loss",
                                         r_cut=(grid.q_min, grid.q_max), n_z=48)
        assert err < 0.03 * abs(mean)
        assert abs(mean - red) < 3.5 * err, (i, mean, red, err)


def test_fractional_reduction_differs_from_absolute_at_the_same_mean_width():
    """The fractional and absolute smearings are different functions: with
    sigma_E equal to w E_in at the observed momentum they still differ by
    more than the quadrature error, so the pin above distinguishes them."""
    q = np.geomspace(1e-3, 40, 128)
    d = lambda x: 0.5 * np.exp(-np.asarray(x) / 1.5)
    p1, w = 2.0, 0.3
    a = ref.two_body_cm_fractional(p1, (0, 0, 0, 0), d(p1), d, d, d, (0, 0, 0, 0), w, n_z=24)
    b = ref.two_body_cm_smeared(p1, (0, 0, 0, 0), d(p1), d, d, d, (0, 0, 0, 0), w * 3.0, n_omega=24)
    assert abs(a - b) > 1e-3 * abs(a)


def test_narrow_fractional_width_approaches_exact_delta():
    grid = Grid(16, 0.01, 30.0, True)
    proc = Process("pp", (0, 0), (0, 0), 1.0, 0.01, 100_000, 5, 0.5, 50, width_mode=WIDTH_FRACTIONAL,
                   width=0.003)
    prob = Problem(grid, (Species("phi", STAT_MB, 0.0),), (proc,), seed=14)
    q = col.grid_q(grid)
    f = (0.5 * np.exp(-q / 1.5))[None, :]
    si = side_integrals(prob)[0]
    i = 9
    mean, err, *_ = col.evaluate_task(prob, 0, si, i, 1, f, 0.0, vegas.uniform_edges(6, 50), 0)
    cf = ref.loss_massless_mb(q[i], 0.5, 1.5)
    assert abs(mean - cf) < 3.5 * err + 2e-3 * cf


def test_controller_rule():
    p = Process("pp", (0, 0), (0, 0), width_mode=WIDTH_ADAPTIVE, width=0.01, width_rel_lo=1e-3,
                width_rel_hi=1e-2, width_factor=2.0, width_min=2e-3, width_max=0.03)
    assert ow.adapt(0.01, 5e-4, p) == 0.005           # below the lower threshold: narrower
    assert ow.adapt(0.01, 2e-2, p) == 0.02            # above the upper threshold: wider
    assert ow.adapt(0.01, 5e-3, p) == 0.01            # in between: kept
    assert ow.adapt(0.003, 1e-4, p) == 2e-3           # clamped below
    assert ow.adapt(0.02, 1.0, p) == 0.03             # clamped above
    assert ow.adapt(0.01, None, p) == 0.01            # undefined error: kept
    assert ow.adapt(0.01, 1.0, replace(p, width_mode=WIDTH_FRACTIONAL)) == 0.01


def test_relative_error_of_equal_independent_tasks():
    """T equal tasks of mean m and error e: the summed rate has relative
    error e / (m sqrt(T))."""
    T, m, e = 16, 3.0, 0.2
    assert np.isclose(ow.relative_error(np.full(T, m), np.full(T, e)), e / (m * np.sqrt(T)), rtol=1e-14)
    assert ow.relative_error([], []) is None
    assert ow.relative_error([0.0, 0.0], [1.0, 1.0]) is None


def test_sweep_adapts_width_by_budget():
    """Small budget (relative error above the upper threshold): w widens
    every sweep until the clamp; large budget (below the lower one): w narrows."""
    grid = Grid(6, 0.05, 20.0, True)
    sp = (Species("phi", STAT_MB, 0.0),)
    q = col.grid_q(grid)
    f = (0.5 * np.exp(-q / 1.5))[None, :]
    for neval, rlo, rhi, want in ((200, 1e-5, 1e-4, "wider"), (4000, 0.5, 0.9, "narrower")):
        proc = Process("pp", (0, 0), (0, 0), 1.0, 0.01, neval, 1, 0.5, 20, width_mode=WIDTH_ADAPTIVE,
                       width=0.01, width_rel_lo=rlo, width_rel_hi=rhi, width_factor=1.5, width_min=0.004,
                       width_max=0.03)
        prob = Problem(grid, sp, (proc,), seed=15)
        st = col.State()
        ws = []
        for _ in range(4):
            col.collision(prob, f, 0.0, st)
            ws.append(st.widths[0])
        if want == "wider":
            assert ws == [0.015, 0.0225, 0.03, 0.03]
        else:
            assert np.allclose(ws, [0.01 / 1.5, 0.01 / 2.25, 0.004, 0.004])
