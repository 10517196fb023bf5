"""Pins of the oracle's grid-level assembly C_a(p_i) = sum_S n_S^a (gain - loss)
(Eq. (7), (8)) through the conservation laws of the collision term.

``collision()`` itself is run over a whole grid and its output integrated
over momentum space, n-weighted (number) and E-weighted (energy):

    R_N = Int q^2 C(q) dq / (2 pi^2),   R_E = Int q^2 E(q) C(q) dq / (2 pi^2),

by the trapezoid rule in ln q on the log grid (the "sum_i C_i q_i^2 dq_i" of a
conservation check), so R = sum_i W_i C_i with positive W_i and its MC error
is sqrt(sum_i W_i^2 err_i^2).

  * 2 -> 2 (Sec. 5C, Fig. 3): number and energy are conserved.  Under the
    Gaussian of Eq. (11) number conservation stays exact (the integrand is
    symmetric under exchanging the initial and final pairs, and the Gaussian
    is even in E_in - E_out); energy picks up a bias of relative order
    (sigma_E / T)^2, T the momentum scale of f (the Gaussian's second moment
    times the variation of the statistical factors).
  * 2 <-> 3 (Sec. 2C, Sec. 5D, Fig. 4): energy is conserved by
    2 C_2 + 3 C_3 and not by C_3 alone.

Bounds: 3 standard errors, plus the quadrature and grid-truncation error
(the integrated legs stop at q_max and the observed momentum is sampled on
the grid; bounded here by the quadrature's error on a closed-form integrand
of the same shape on the same grid, times 10), plus the Gaussian bias above
for energy.  A slip in the signs or multiplicities of the assembly moves a
residual to the size of the scale sum_i W_i (gain_i + loss_i).
"""
import numpy as np
import pytest
from scipy.special import gamma

from oracle import collision as col
from oracle import reference as ref
from oracle.tasks import side_integrals
from workloads import STAT_BE, STAT_MB, Grid, Problem, Process, Species

from _oracle_pool import collision_sweeps


def _weights(prob, m=0.0):
    """W_i of R_N and R_E: the trapezoid rule in ln q on the log grid,
    Int q^2 g dq = Int q^3 g d ln q ~ sum_i h q_i^3 g_i (halved at the ends),
    whose weights are all positive; the integrands vanish at both ends of the
    grid, where the rule converges fastest."""
    q = col.grid_q(prob.grid)
    h = np.log(q[1] / q[0])
    w = h * q ** 3 / (2 * np.pi ** 2)
    w[0] *= 0.5
    w[-1] *= 0.5
    return w, w * np.sqrt(q * q + m * m)


def _quadrature_bound(prob, T):
    """Relative error of that rule, including the truncation at the grid's
    ends, on q^2 E^k e^{-q/T} for k = 0 (number) and k = 1 (massless energy)
    against their closed forms Int_0^inf q^(k+2) e^{-q/T} dq = T^(k+3) (k+2)!."""
    q = col.grid_q(prob.grid)
    Wn, We = _weights(prob)
    g = np.exp(-q / T)
    exact = lambda k: T ** (k + 3) * gamma(k + 3) / (2 * np.pi ** 2)
    return max(abs(Wn @ g / exact(0) - 1.0), abs(We @ g / exact(1) - 1.0))


def _sides(prob, detail):
    """Per side S of the observed leg: n_S (gain - loss), n_S^2 (err_g^2 +
    err_l^2) and n_S (gain + loss) per grid point, from the per-task detail."""
    n = prob.grid.n
    C, V, S = np.zeros((2, n)), np.zeros((2, n)), np.zeros((2, n))
    for k, si in enumerate(side_integrals(prob)):
        for i in range(n):
            g, eg = detail[(k * n + i) * 2]
            l, el = detail[(k * n + i) * 2 + 1]
            C[si.side, i] += si.mult * (g - l)
            V[si.side, i] += si.mult ** 2 * (eg * eg + el * el)
            S[si.side, i] += si.mult * (g + l)
    return C, V, S


@pytest.mark.parametrize("stat", [STAT_MB, STAT_BE], ids=["mb", "be"])
def test_2to2_conserves_number_and_energy(stat):
    """m = 1, f = equilibrium-like e^{-E} (MB: 0.5 e^{-E}; BE: 1/(e^E - 1)) plus
    a bump 0.2 e^{-(q-2)^2/(2 0.5^2)}, so that C is far from zero; one
    training sweep, then the measured sweep on the trained maps."""
    m, T, sig = 1.0, 1.0, 0.05
    grid = Grid(32, 0.01, 15.0, True)
    proc = Process("pp", (0, 0), (0, 0), 1.0, sig, 20_000, 3, 0.5, 50)
    prob = Problem(grid, (Species("phi", stat, m),), (proc,), seed=21)
    q = col.grid_q(grid)
    E = np.sqrt(q * q + m * m)
    base = 0.5 * np.exp(-E / T) if stat == STAT_MB else 1.0 / np.expm1(E / T)
    f = (base + 0.2 * np.exp(-(q - 2.0) ** 2 / (2 * 0.5 ** 2)))[None, :]
    C, err, detail = collision_sweeps([prob, prob.with_budget(100_000, 3)], f)
    Wn, We = _weights(prob, m)
    _, _, S = _sides(prob, detail)
    quad = 10.0 * _quadrature_bound(prob, T)
    for W, bias in ((Wn, 0.0), (We, (sig / T) ** 2)):
        R = W @ C[0]
        sR = np.sqrt(np.sum((W * err[0]) ** 2))
        scale = W @ S.sum(axis=0)
        assert sR < 0.02 * scale                       # the check has power
        assert abs(R) <= 3.0 * sR + (quad + bias) * scale, (R, sR, scale)


def test_2to3_energy_conserved_by_both_sides_not_by_c3_alone():
    """Massless MB f = A e^{-q/T}, A = 0.25 (out of chemical equilibrium): the
    energy residual of C = 2 C_2 + 3 C_3 as assembled by ``collision()`` is
    within its bounds of zero, while that of the 3-leg side alone is many
    standard errors from zero (the paper: about 1% against about 40%)."""
    A, T, sig = 0.25, 1.0, 0.1
    grid = Grid(20, 0.05, 20.0, True)
    proc = Process("p23", (0, 0), (0, 0, 0), 1.0, sig, 10_000, 3, 0.5, 50)
    prob = Problem(grid, (Species("phi", STAT_MB, 0.0),), (proc,), seed=22)
    q = col.grid_q(grid)
    f = (A * np.exp(-q / T))[None, :]
    C, err, detail = collision_sweeps([prob, prob, prob.with_budget(100_000, 3)], f)
    _, We = _weights(prob)
    Cs, Vs, S = _sides(prob, detail)
    assert np.allclose(Cs.sum(axis=0), C[0], rtol=1e-12, atol=0.0)
    scale = We @ S.sum(axis=0)
    R = We @ C[0]
    sR = np.sqrt(np.sum((We * err[0]) ** 2))
    R3 = We @ Cs[1]
    s3 = np.sqrt(np.sum(We ** 2 * Vs[1]))
    quad = 10.0 * _quadrature_bound(prob, T)
    assert sR < 0.02 * scale
    assert abs(R) <= 3.0 * sR + (quad + (sig / T) ** 2) * scale, (R, sR, scale)
    assert abs(R3) > 8.0 * s3, (R3, s3)
    assert abs(R3) > 0.2 * (We @ S[1])


def test_2to2_collision_is_twice_the_side_integral():
    """phi phi -> phi phi takes one side with multiplicity 2 (Eq. (8) and the
    2 C_BW of Sec. 4): C(p_i) from ``collision()`` equals 2 (gain - loss) of
    the independent centre-of-mass quadrature with the same Gaussian (width
    0.2) and the same restriction of the integrated legs, within 3.5 sigma."""
    m, sig = 0.5, 0.2
    grid = Grid(16, 0.01, 30.0, True)
    proc = Process("pp", (0, 0), (0, 0), 1.0, sig, 40_000, 4, 0.5, 50)
    prob = Problem(grid, (Species("phi", STAT_BE, m),), (proc,), seed=23)
    q = col.grid_q(grid)
    f = (1.0 / np.expm1(np.sqrt(q * q + m * m)) + 0.3 * np.exp(-(q - 3.0) ** 2 / (2 * 0.5 ** 2)))[None, :]
    pts = (6, 9)
    C, err, _ = col.collision(prob, f, 0.0, col.State(), "f64", points=pts)
    d = col.distributions(prob, f, 0.0)[0]
    for i in pts:
        red = [ref.two_body_cm_smeared(q[i], (m,) * 4, f[0, i], d, d, d, (1.0,) * 4, sig, term=term,
                                       r_cut=(grid.q_min, grid.q_max), n_omega=24)
               for term in ("gain", "loss")]
        expect = 2.0 * (red[0] - red[1])
        assert err[0, i] < 0.1 * (red[0] + red[1])
        assert abs(C[0, i] - expect) < 3.5 * err[0, i], (i, C[0, i], expect, err[0, i])
    assert np.all(C[0, [i for i in range(grid.n) if i not in pts]] == 0.0)
