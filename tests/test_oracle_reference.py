"""Pins of the Monte Carlo oracle against exact-energy reductions of the
2 -> 2 collision integral (Sec. 4, App. B) and a closed form."""
import numpy as np
import pytest

from oracle import collision as col
from oracle import reference as ref
from oracle import vegas
from oracle.spline import Distribution
from oracle.tasks import side_integrals
from workloads import STAT_BE, STAT_MB, Grid, Problem, Process, Species


def _bose_bump(q, m, T=1.0):
    return 1.0 / np.expm1(np.sqrt(q * q + m * m) / T) + 0.3 * np.exp(-(q - 3.0) ** 2 / (2 * 0.5 ** 2))


def test_closed_form_equals_cm_reduction():
    A, T = 0.5, 1.5
    mb = lambda q: A * np.exp(-np.asarray(q) / T)
    for p1 in (0.2, 1.0, 4.0):
        cf = ref.loss_massless_mb(p1, A, T)
        cm = ref.two_body_cm(p1, (0, 0, 0, 0), mb(p1), mb, mb, mb, (0, 0, 0, 0), term="loss")
        assert np.isclose(cm, cf, rtol=1e-10)
        # detailed balance with exact energy conservation: gain = loss
        cg = ref.two_body_cm(p1, (0, 0, 0, 0), mb(p1), mb, mb, mb, (0, 0, 0, 0), term="gain")
        assert np.isclose(cg, cf, rtol=1e-10)


@pytest.mark.parametrize("masses", [(1, 1, 1, 1), (0.5, 0.5, 0.5, 0.5), (1, 0.3, 1, 0.3),
                                    (0.2, 0.7, 0.4, 1.1)])
def test_paper_semi_analytic_matches_cm_reduction(masses):
    """The paper's backward term C_BW (Eq. (18)-(19), App. B, as printed) and
    the independent centre-of-mass reduction agree: C_BW is the
    single-position gain term (without the multiplicity)."""
    q = np.geomspace(1e-3, 40, 128)
    ds = [Distribution(q, _bose_bump(q, m), STAT_BE, m) for m in masses]
    for p1 in (0.3, 2.0):
        f1 = ds[0](np.array([p1]))[0]
        cm = ref.two_body_cm(p1, masses, f1, ds[1], ds[2], ds[3], (1, 1, 1, 1), term="gain")
        pb = ref.paper_backward_term(p1, masses, f1, ds[1], ds[2], ds[3], (1, 1, 1, 1))
        assert np.isclose(pb, cm, rtol=1e-3)


@pytest.mark.parametrize("case", ["mb_massless_loss", "be_massive_gain", "be_massive_loss"])
def test_mc_matches_gaussian_smeared_reduction(case):
    """The Monte Carlo estimate of a 2 -> 2 term equals the same term computed
    by quadrature with the Gaussian of Eq. (11), within 3.5 sigma; the width is
    wide (0.2) so that a modest budget suffices, and the restriction of the
    integrated legs to [q_min, q_max] is applied to both."""
    if case == "mb_massless_loss":
        m, stat, eta, term, pts = 0.0, STAT_MB, 0.0, 1, (4, 8)
        fq = lambda q: 0.5 * np.exp(-q / 1.5)
    else:
        m, stat, eta, term, pts = 0.5, STAT_BE, 1.0, (0 if case.endswith("gain") else 1), (6, 9)
        fq = lambda q: _bose_bump(q, 0.5)
    grid = Grid(16, 0.01, 30.0, True)
    prob = Problem(grid, (Species("phi", stat, m),),
                   (Process("pp", (0, 0), (0, 0), 1.0, 0.2, 40_000, 4, 0.5, 50),), seed=11)
    q = col.grid_q(grid)
    f = fq(q)[None, :]
    dists = col.distributions(prob, f, 0.0)
    si = side_integrals(prob)[0]
    for i in pts:
        mean, err, *_ = col.evaluate_task(prob, 0, si, i, term, f, 0.0,
                                            vegas.uniform_edges(6, 50), 0, "f64", dists)
        d = dists[0]
        red = ref.two_body_cm_smeared(q[i], (m, m, m, m), f[0, i], d, d, d, (eta,) * 4, 0.2,
                                      term="gain" if term == 0 else "loss",
                                      r_cut=(grid.q_min, grid.q_max), n_omega=24)
        assert err < 0.03 * abs(mean)
        assert abs(mean - red) < 3.5 * err, (i, mean, red, err)


def test_mc_narrow_gaussian_approaches_exact_delta():
    """At the workloads' narrow width (0.01) the Monte Carlo term approaches
    the exact-delta closed form (bias O(sigma^2) below the MC error)."""
    grid = Grid(16, 0.01, 30.0, True)
    prob = Problem(grid, (Species("phi", STAT_MB, 0.0),),
                   (Process("pp", (0, 0), (0, 0), 1.0, 0.01, 100_000, 5, 0.5, 50),), seed=12)
    q = col.grid_q(grid)
    f = (0.5 * np.exp(-q / 1.5))[None, :]
    si = side_integrals(prob)[0]
    i = 9
    mean, err, *_ = col.evaluate_task(prob, 0, si, i, 1, f, 0.0, vegas.uniform_edges(6, 50), 0)
    cf = ref.loss_massless_mb(q[i], 0.5, 1.5)
    assert abs(mean - cf) < 3.5 * err + 2e-3 * cf
