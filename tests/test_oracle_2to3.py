"""Pins of the oracle's five-leg side integrals (2 <-> 3, Sec. 2C, Sec. 5D)
and of the decomposition C = 2 C_2 + 3 C_3 through energy conservation."""
import numpy as np
import pytest

from oracle import collision as col
from oracle import reference as ref
from oracle import vegas
from oracle.tasks import side_integrals
from workloads import STAT_MB, Grid, Problem, Process, Species

A, T = 0.5, 1.0


def closed_c2(p):   # massless MB, |M|^2 = 1: Phi_3 = s / (256 pi^3)
    return A * A * T ** 3 * np.exp(-p / T) / (512 * np.pi ** 5)


def closed_c3(p):   # massless MB: Phi_2 = 1 / (8 pi)
    return A ** 3 * T ** 4 * np.exp(-p / T) / (256 * np.pi ** 5 * p)


def test_reductions_reach_massless_closed_forms():
    for p in (0.5, 2.0):
        assert np.isclose(ref.loss_2to3_c2_mb(p, 0.0, A, T, 0.002), closed_c2(p), rtol=1e-4)
        assert np.isclose(ref.loss_2to3_c3_mb(p, 0.0, A, T, 0.002), closed_c3(p), rtol=1e-4)


def test_decomposition_conserves_energy():
    """For massless MB legs f = A e^{-p/T} (out of chemical equilibrium when
    A != 1) the per-sample detailed balance gives C_2 = (A - 1) loss_2 and
    C_3 = (1/A - 1) loss_3 with the exact delta.  Energy conservation holds
    for 2 C_2 + 3 C_3 and fails for C_3 alone (Sec. 2C, Sec. 5D)."""
    p = np.geomspace(1e-4, 80, 4000)
    wts = np.gradient(p)
    e2 = np.sum(4 * np.pi * p ** 2 * p * (A - 1) * closed_c2(p) * wts)
    e3 = np.sum(4 * np.pi * p ** 2 * p * (1 / A - 1) * closed_c3(p) * wts)
    assert abs(2 * e2 + 3 * e3) < 1e-3 * abs(3 * e3)
    assert abs(3 * e3) > 0.5 * abs(2 * e2)          # C_3 alone is far from zero


@pytest.mark.parametrize("side,i", [(0, 16), (0, 24), (1, 16), (1, 24)])
def test_mc_matches_reduction_massive(side, i):
    """Massive (m = 1) MB 2 -> 3: the Monte Carlo loss of each side integral
    matches its Gaussian-smeared reduction (width 0.2) within 3.5 sigma."""
    m, sigma = 1.0, 0.2
    grid = Grid(48, 0.01, 30.0, True)
    prob = Problem(grid, (Species("phi", STAT_MB, m),),
                   (Process("p", (0, 0), (0, 0, 0), 1.0, sigma, 60_000, 4),), seed=5)
    q = col.grid_q(grid)
    f = (A * np.exp(-np.sqrt(q * q + m * m) / T))[None, :]
    si = side_integrals(prob)[side]
    mean, err, *_ = col.evaluate_task(prob, side, si, i, 1, f, 0.0, vegas.uniform_edges(9, 50), 0)
    red = (ref.loss_2to3_c2_mb if side == 0 else ref.loss_2to3_c3_mb)(q[i], m, A, T, sigma)
    assert err < 0.05 * mean
    assert abs(mean - red) < 3.5 * err


def test_side_selection_keeps_roles_and_multiplicities():
    """sides = 1 / 2 keep only the side integrals with the observed leg
    initial / final (the paper's C_3 alone, Sec. 5D), with the roles and
    multiplicities they have in the full decomposition; a process with equal
    initial and final species has no final-side integral to keep."""
    from dataclasses import replace
    prob = Problem(Grid(8, 0.1, 10.0, True), (Species("phi", STAT_MB, 1.0),),
                   (Process("p", (0, 0), (0, 0, 0), 1.0, 0.1, 100, 1),))
    full = side_integrals(prob)
    assert [s.side for s in full] == [0, 1] and [s.mult for s in full] == [2, 3]
    for keep in (1, 2):
        sel = side_integrals(replace(prob, processes=(replace(prob.processes[0], sides=keep),)))
        assert sel == [s for s in full if s.side == keep - 1]
    sym = replace(prob, processes=(Process("q", (0, 0), (0, 0), sides=2),))
    assert side_integrals(sym) == []
