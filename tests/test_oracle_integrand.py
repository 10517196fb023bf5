"""Pins of the oracle's per-sample integrand: roles (App. A), kinematics,
statistical factors (Eq. (5)), weights and the expansion scaling (Sec. 3E)."""
from dataclasses import replace

import numpy as np
import pytest

from oracle import collision as col
from oracle import philox, vegas
from oracle.tasks import SIDE_IN, SIDE_OUT, side_integrals
from workloads import (STAT_BE, STAT_FD, STAT_MB, Expansion, Grid, Problem, Process,
                       Species)


def _problem(sp_in, sp_out, species, sigma=0.05, grid=Grid(16, 0.02, 15.0, True), **kw):
    return Problem(grid, tuple(species), (Process("p", sp_in, sp_out, 1.3, sigma, 1000, 1),), seed=3, **kw)


def test_roles_and_multiplicities():
    bos = Species("phi", STAT_BE, 1.0)
    si = side_integrals(_problem((0, 0), (0, 0, 0), [bos]))
    assert [(s.side, s.species, s.mult, s.obs, s.cons, s.integrated) for s in si] == [
        (SIDE_IN, 0, 2, 0, 1, (2, 3, 4)),    # C_2: observed on the 2-particle side
        (SIDE_OUT, 0, 3, 2, 0, (1, 3, 4)),   # C_3: conserved stays on the fewer side
    ]
    si = side_integrals(_problem((0, 0), (0, 0), [bos]))
    assert [(s.side, s.mult, s.obs, s.cons) for s in si] == [(SIDE_IN, 2, 0, 1)]
    A, B = Species("A", STAT_BE, 1.0), Species("B", STAT_FD, 0.3)
    si = side_integrals(_problem((0, 1), (0, 1), [A, B]))
    assert [(s.side, s.species, s.mult, s.obs, s.cons) for s in si] == [
        (SIDE_IN, 0, 1, 0, 1), (SIDE_IN, 1, 1, 1, 0)]
    si = side_integrals(_problem((0, 0, 0), (1, 1), [A, B]))
    assert [(s.side, s.species, s.mult, s.obs, s.cons, s.integrated) for s in si] == [
        (SIDE_IN, 0, 3, 0, 3, (1, 2, 4)), (SIDE_OUT, 1, 2, 3, 4, (0, 1, 2))]
    # a decay: the fewer side holds only the observed leg -> fallback
    si = side_integrals(_problem((0,), (1, 1), [A, B]))
    assert [(s.side, s.species, s.mult, s.obs, s.cons, s.integrated) for s in si] == [
        (SIDE_IN, 0, 1, 0, 1, (2,)), (SIDE_OUT, 1, 2, 1, 0, (2,))]


def _samples(D, N=4000, seed=9):
    return philox.uniforms(seed, 0, 0, 0, N, D, "f64")


@pytest.mark.parametrize("sp_in,sp_out", [((0, 0), (0, 0)), ((0, 0), (0, 0, 0)),
                                          ((0, 0, 0), (0, 0)), ((0, 0), (0, 0, 0, 0))])
def test_momentum_conservation_and_on_shell(sp_in, sp_out):
    prob = _problem(sp_in, sp_out, [Species("phi", STAT_BE, 0.7)])
    for si in side_integrals(prob):
        y = _samples(si.dim)
        mom, E, qcom, jac = col.kinematics(prob, si, 5, np.array([0.7]), 1.0, y)
        p_in = sum(mom[k] for k in range(si.n) if si.is_in(k))
        p_out = sum(mom[k] for k in range(si.n) if not si.is_in(k))
        assert np.allclose(p_in, p_out, atol=1e-12)
        assert np.allclose(E ** 2 - np.sum(mom ** 2, axis=2), 0.49, atol=1e-10)
        grid = col.grid_q(prob.grid)
        assert np.allclose(mom[si.obs], [0, 0, grid[5]])


@pytest.mark.parametrize("stat,eta", [(STAT_MB, 0.0), (STAT_BE, 1.0), (STAT_FD, -1.0)])
@pytest.mark.parametrize("sp_in,sp_out", [((0, 0), (0, 0)), ((0, 0), (0, 0, 0)),
                                          ((0, 0, 0), (0, 0))])
def test_detailed_balance_per_sample(stat, eta, sp_in, sp_out):
    """At equilibrium f/(1 + eta f) = exp(-(E - mu)/T), so per sample
    gain/loss = exp((sum_own E - sum_other E)/T + (n_other - n_own) mu/T);
    this fixes which legs carry f and which (1 + eta f) in each term."""
    T, mu, m = 1.1, -0.2, 0.8
    prob = _problem(sp_in, sp_out, [Species("phi", stat, m)])
    feq = lambda q: 1.0 / (np.exp((np.sqrt(np.asarray(q) ** 2 + m * m) - mu) / T) - eta)
    grid = col.grid_q(prob.grid)
    for si in side_integrals(prob):
        y = _samples(si.dim)
        i = 6
        g = col.integrand(prob, si, 0, i, feq(grid[i]), [feq], np.array([m]), 1.0, y)
        l = col.integrand(prob, si, 1, i, feq(grid[i]), [feq], np.array([m]), 1.0, y)
        _, E, _, _ = col.kinematics(prob, si, i, np.array([m]), 1.0, y)
        own = [k for k in range(si.n) if si.is_in(k) == (si.side == SIDE_IN)]
        oth = [k for k in range(si.n) if k not in own]
        expo = (E[own].sum(0) - E[oth].sum(0)) / T + (len(oth) - len(own)) * mu / T
        keep = l > 1e-300
        assert keep.sum() > 100
        assert np.allclose(g[keep] / l[keep], np.exp(expo[keep]), rtol=1e-9)


def test_rotation_and_permutation_invariance():
    prob = _problem((0, 0), (0, 0, 0), [Species("phi", STAT_BE, 1.0)])
    q = col.grid_q(prob.grid)
    f = 0.3 * np.exp(-q / 1.2) + 0.05 * np.exp(-(q - 2) ** 2)
    d = col.distributions(prob, f[None, :], 0.0)
    si = side_integrals(prob)[1]
    y = _samples(si.dim)
    w0 = col.integrand(prob, si, 0, 4, f[4], d, np.array([1.0]), 1.0, y)
    yr = y.copy()
    yr[:, 2::3] = (yr[:, 2::3] + 0.3137) % 1.0      # common azimuthal rotation
    wr = col.integrand(prob, si, 0, 4, f[4], d, np.array([1.0]), 1.0, yr)
    assert np.allclose(wr, w0, rtol=1e-9, atol=1e-300)
    yp = y.copy()
    assert si.integrated == (1, 3, 4)
    yp[:, 3:6], yp[:, 6:9] = y[:, 6:9], y[:, 3:6]   # swap legs 3 and 4 (same side, same species)
    wp = col.integrand(prob, si, 0, 4, f[4], d, np.array([1.0]), 1.0, yp)
    assert np.allclose(wp, w0, rtol=1e-9, atol=1e-300)


def test_expansion_is_a_rescaling():
    """With comoving grid q at scale factor a the integral equals the a = 1
    integral on the grid q/a with the same grid values (Sec. 3E: p = q/a,
    d^3p = d^3q/a^3, q_cons = |p_cons| a): same samples, same result."""
    sp = [Species("phi", STAT_BE, 0.6)]
    g2 = Grid(12, 0.04, 16.0, True)
    g1 = Grid(12, 0.02, 8.0, True)
    pa = replace(_problem((0, 0), (0, 0, 0), sp, grid=g2), expansion=Expansion(1.0, 1.0))
    p1 = _problem((0, 0), (0, 0, 0), sp, grid=g1)
    q = col.grid_q(g2)
    f = (0.25 * np.exp(-np.sqrt(q * q / 4 + 0.36) / 0.9))[None, :]
    t = 4.0                                        # a = (t/t0)^(1/2) = 2
    assert col.scale_factor(pa, t) == 2.0
    for k, si in enumerate(side_integrals(pa)):
        for term in (0, 1):
            e = vegas.uniform_edges(si.dim, 50)
            ra = col.evaluate_task(pa, k, si, 5, term, f, t, e, 0)
            r1 = col.evaluate_task(p1, k, si, 5, term, f, t, e, 0)
            assert ra[0] > 0 and np.isclose(ra[0], r1[0], rtol=1e-9)
