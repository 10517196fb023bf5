"""Energy bookkeeping of number-changing processes on the GPU path (Sec. 2C,
Sec. 5D, Fig. 4): C = 2 C_2 + 3 C_3 of a 2 <-> 3 process conserves energy,
C_3 alone does not; and the same holds for the densities of an evolution.

The energy residual R_E = Int q^2 E C dq / (2 pi^2) is taken with the
trapezoid rule in ln q on the log grid (as the oracle's conservation pins
do); its MC error follows from the per-point errors.  Every number comes
from the library through the C ABI; the side contributions are assembled
from its per-task results with the multiplicities of Eq. (7).
"""
import numpy as np
import pytest

import workloads as W
from tests._helpers import side_integrals

pytestmark = pytest.mark.gpu


def _log_trapezoid(q, m=0.0):
    h = np.log(q[1] / q[0])
    w = h * q ** 3 / (2 * np.pi ** 2)
    w[0] *= 0.5
    w[-1] *= 0.5
    return w * np.sqrt(q * q + m * m)


def test_energy_residual_of_both_sides_vanishes_not_c3_alone():
    """Massless MB f = A e^{-q/T}, A = 0.25 (out of chemical equilibrium),
    sigma_E = 0.1, FP32: after a training sweep the residual of C is
    within 3 standard errors + the Gaussian bias (sigma/T)^2 + the rule's
    error of zero, and C_3 alone is many standard errors from zero."""
    import torch

    from oracle.collision import grid_q
    from paper_2603_28848_gb300 import Collision
    A, T, sig = 0.25, 1.0, 0.1
    grid = W.Grid(32, 0.05, 20.0, True)
    proc = W.Process("p23", (0, 0), (0, 0, 0), 1.0, sig, 1_000_000, 3, 0.5, 50)
    prob = W.Problem(grid, (W.Species("phi", W.STAT_MB, 0.0),), (proc,), seed=41)
    q = grid_q(grid)
    f = torch.tensor((A * np.exp(-q / T))[None, :], dtype=torch.float64, device="cuda")
    big = prob
    col2 = Collision(big, W.PREC_FP32)
    col2.eval(f, 0.0)                       # trains the maps
    C, err = col2.eval(f, 0.0)
    col2.check()
    mean, terr = col2.task_results()
    col2.close()
    C, err = C.cpu().numpy()[0], err.cpu().numpy()[0]
    n = grid.n
    Cs, Vs, Ss = np.zeros((2, n)), np.zeros((2, n)), np.zeros((2, n))
    for k, si in enumerate(side_integrals(big)):
        for i in range(n):
            g, l = (k * n + i) * 2, (k * n + i) * 2 + 1
            Cs[si.side, i] += si.mult * (mean[g] - mean[l])
            Vs[si.side, i] += si.mult ** 2 * (terr[g] ** 2 + terr[l] ** 2)
            Ss[si.side, i] += si.mult * (abs(mean[g]) + abs(mean[l]))
    assert np.allclose(Cs.sum(axis=0), C, rtol=1e-9, atol=1e-300)
    We = _log_trapezoid(q)
    scale = We @ Ss.sum(axis=0)
    R, sR = We @ C, np.sqrt(np.sum((We * err) ** 2))
    R3, s3 = We @ Cs[1], np.sqrt(np.sum(We ** 2 * Vs[1]))
    assert sR < 0.02 * scale
    assert abs(R) <= 3.0 * sR + (0.005 + (sig / T) ** 2) * scale, (R / scale, sR / scale)
    assert abs(R3) > 20.0 * s3 and abs(R3) > 0.3 * (We @ Ss[1]), (R3, s3)


def test_c3_alone_evolution_does_not_conserve_energy():
    """Euler steps of the 2 <-> 3 workload (BE, m = 1, f0 = 0.2 e^{-E/0.7},
    reduced budget), each as long as the bound of Eq. (16) allows, from the
    same f0: with both sides (C = 2 C_2 + 3 C_3) the number density grows and
    the energy density stays within 2% (the paper: about 1%); with the 3-leg
    side alone the energy density moves by more than 10% (the paper: about
    40%) and by ten times more than with both sides."""
    from dataclasses import replace

    from paper_2603_28848_gb300 import evolve
    prob, f0 = W.c3_cannibal_2to3(n=48, neval=40_000, nitn=3)
    run = lambda p: evolve.run(p, f0, steps=12, every=4, precision=W.PREC_FP32, t0=0.0, dt=1e9, autotune=False,
                               method="euler")
    full = run(prob)
    only3 = run(replace(prob, processes=(replace(prob.processes[0], sides=2),)))
    e_full = abs(full["final_rel_change_rho"][0])
    e_c3 = abs(only3["final_rel_change_rho"][0])
    assert full["max_abs_dlogf"] > 0.5 and only3["max_abs_dlogf"] > 0.5
    assert full["final_rel_change_n"][0] > 0.002                      # number changing
    assert e_full < 0.02, e_full
    assert e_c3 > 0.1 and e_c3 > 10 * e_full, (e_full, e_c3)
