"""Pins of the density diagnostics: exact for a cubic f, the massless
Maxwell-Boltzmann closed forms (incomplete gamma functions) on a fine grid,
and the a^-3 / a^-4 scaling of n and rho for massless particles."""
import numpy as np
from scipy.special import gamma, gammainc

from oracle import moments as om
from oracle.collision import grid_q
from workloads import STAT_MB, Expansion, Grid, Problem, Process, Species


def _prob(grid, mass=0.0, expansion=None):
    return Problem(grid, (Species("phi", STAT_MB, mass),), (Process("pp", (0, 0), (0, 0)),),
                   expansion=expansion)


def test_cubic_f_is_exact():
    grid = Grid(9, 0.5, 4.0, True)
    prob = _prob(grid)
    q = grid_q(grid)
    c = (0.3, -0.2, 0.05, 0.01)
    f = (c[0] + c[1] * q + c[2] * q ** 2 + c[3] * q ** 3)[None, :]
    n, _ = om.moments(prob, f, 0.0)
    P = lambda x: sum(ck * x ** (k + 3) / (k + 3) for k, ck in enumerate(c))
    assert np.isclose(n[0], (P(4.0) - P(0.5)) / (2 * np.pi ** 2), rtol=1e-13)


def test_massless_mb_closed_forms():
    """f = A e^{-q/T}: Int q^k e^{-q/T} dq = T^{k+1} Gamma(k+1) [P(k+1, q/T)]."""
    A, T = 0.7, 1.3
    grid = Grid(600, 1e-3, 40.0, True)
    prob = _prob(grid)
    q = grid_q(grid)
    n, rho = om.moments(prob, (A * np.exp(-q / T))[None, :], 0.0)
    inc = lambda k: T ** (k + 1) * gamma(k + 1) * (gammainc(k + 1, 40.0 / T) - gammainc(k + 1, 1e-3 / T))
    assert np.isclose(n[0], A * inc(2) / (2 * np.pi ** 2), rtol=1e-7)
    assert np.isclose(rho[0], A * inc(3) / (2 * np.pi ** 2), rtol=1e-7)


def test_expansion_scaling_massless():
    grid = Grid(64, 0.01, 20.0, True)
    q = grid_q(grid)
    f = (1.0 / np.expm1(q))[None, :]
    n1, r1 = om.moments(_prob(grid, expansion=Expansion(1.0, 1.0)), f, 1.0)
    n4, r4 = om.moments(_prob(grid, expansion=Expansion(1.0, 1.0)), f, 4.0)     # a = 2
    assert np.isclose(n4[0], n1[0] / 8.0, rtol=1e-14)
    assert np.isclose(r4[0], r1[0] / 16.0, rtol=1e-14)
