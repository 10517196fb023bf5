"""Pins of the s-dependent matrix element |M|^2 = coupling^2 P(s): the
invariant of each sample against the two-particle formula, the default
(constant) reproducing the plain weight, and the Monte Carlo term with
P(s) = s against the independent centre-of-mass quadrature."""
from dataclasses import replace

import numpy as np
import pytest

from oracle import collision as col
from oracle import philox, vegas
from oracle import reference as ref
from oracle.tasks import side_integrals
from workloads import STAT_BE, STAT_MB, Grid, Problem, Process, Species


def _prob(me=(1.0, 0.0, 0.0, 0.0), m=0.0, stat=STAT_MB, neval=40_000):
    grid = Grid(16, 0.01, 30.0, True)
    proc = Process("pp", (0, 0), (0, 0), 1.0, 0.2, neval, 4, 0.5, 50, me_coef=me)
    return Problem(grid, (Species("phi", stat, m),), (proc,), seed=31)


def test_invariant_matches_two_particle_formula():
    """Two initial legs: s = m1^2 + m2^2 + 2 (E1 E2 - p1 . p2)."""
    prob = _prob(m=0.7)
    si = side_integrals(prob)[0]
    a = 1.0
    m = col.masses(prob, 0.0)
    x = philox.uniforms(prob.seed, 2, 0, 0, 300, si.dim, "f64")
    y, _, _ = vegas.apply_map(vegas.uniform_edges(si.dim, 10), x)
    mom, E, _, _ = col.kinematics(prob, si, 5, m, a, y)
    s = col.invariant_s(si, mom, E)
    ins = [k for k in range(si.n) if si.is_in(k)]
    assert len(ins) == 2
    k1, k2 = ins
    alt = 2 * 0.49 + 2 * (E[k1] * E[k2] - np.sum(mom[k1] * mom[k2], axis=1))
    assert np.allclose(s, alt, rtol=1e-12, atol=1e-12)
    assert np.all(s >= 4 * 0.49 * (1 - 1e-12))      # threshold of two massive particles


def test_constant_default_is_the_plain_weight():
    p0, p1 = _prob(), _prob(me=(2.5, 0.0, 0.0, 0.0))
    q = col.grid_q(p0.grid)
    f = (0.5 * np.exp(-q / 1.5))[None, :]
    dists = col.distributions(p0, f, 0.0)
    si = side_integrals(p0)[0]
    e0 = vegas.uniform_edges(6, 50)
    a = col.evaluate_task(replace(p0, processes=(replace(p0.processes[0], nitn=1, neval=2000),)),
                          0, si, 6, 1, f, 0.0, e0, 0, "f64", dists)
    b = col.evaluate_task(replace(p1, processes=(replace(p1.processes[0], nitn=1, neval=2000),)),
                          0, si, 6, 1, f, 0.0, e0, 0, "f64", dists)
    assert np.isclose(b[0], 2.5 * a[0], rtol=1e-13)


@pytest.mark.parametrize("case", ["mb_massless_loss", "be_massive_gain"])
def test_s_linear_matrix_element_matches_reduction(case):
    if case == "mb_massless_loss":
        m, stat, eta, term, pts = 0.0, STAT_MB, 0.0, 1, (6, 9)
        fq = lambda q: 0.5 * np.exp(-q / 1.5)
    else:
        m, stat, eta, term, pts = 0.5, STAT_BE, 1.0, 0, (6, 9)
        fq = lambda q: 1.0 / np.expm1(np.sqrt(q * q + m * m)) + 0.3 * np.exp(-(q - 3.0) ** 2 / 0.5)
    prob = _prob(me=(0.0, 1.0, 0.0, 0.0), m=m, stat=stat)
    q = col.grid_q(prob.grid)
    f = fq(q)[None, :]
    dists = col.distributions(prob, f, 0.0)
    si = side_integrals(prob)[0]
    d = dists[0]
    for i in pts:
        mean, err, *_ = col.evaluate_task(prob, 0, si, i, term, f, 0.0, vegas.uniform_edges(6, 50), 0, "f64",
                                          dists)
        red = ref.two_body_cm_smeared(q[i], (m, m, m, m), f[0, i], d, d, d, (eta,) * 4, 0.2,
                                      term="gain" if term == 0 else "loss",
                                      r_cut=(prob.grid.q_min, prob.grid.q_max), n_omega=24, me=lambda s: s)
        assert err < 0.03 * abs(mean)
        assert abs(mean - red) < 3.5 * err, (i, mean, red, err)


def test_adjoint_oracle_mass_gradient_through_s():
    """dL/dm of the fixed-sample integral with P(s) = 1 + 0.5 s + 0.1 s^2
    (the invariant depends on the masses through the energies) against
    central differences."""
    import torch
    from oracle import adjoint as adj
    grid = Grid(6, 0.05, 20.0, True)
    proc = Process("pp", (0, 0), (0, 0), 1.0, 0.05, 300, 1, 0.5, 20, me_coef=(1.0, 0.5, 0.1, 0.0))
    prob = Problem(grid, (Species("phi", STAT_BE, 0.8),), (proc,), seed=32)
    q = col.grid_q(grid)
    f0 = (1.0 / np.expm1(np.sqrt(q * q + 0.64)))[None, :]
    maps = {t: vegas.uniform_edges(6, 20) for t in range(2 * grid.n)}
    rng = np.random.default_rng(3)
    v = rng.normal(size=f0.shape)
    C, gf, gm, gl = adj.vjp(prob, f0, 0.0, v, maps, 0)

    def L(mass):
        with torch.no_grad():
            Ct = adj.fixed_sample_C(prob, torch.tensor(f0), torch.tensor([mass], dtype=torch.float64),
                                    torch.tensor([1.0], dtype=torch.float64), 0.0, maps, 0)
        return float((Ct.numpy() * v).sum())

    h = 1e-5
    fd = (L(0.8 * (1 + h)) - L(0.8 * (1 - h))) / (2 * h * 0.8)
    assert abs(fd - gm[0]) <= 1e-4 * abs(gm[0])
