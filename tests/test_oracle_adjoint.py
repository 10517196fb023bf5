"""Pins of the differentiable fixed-sample collision integral (the adjoint's
oracle): it restates the Monte Carlo integrand exactly, and its autograd
gradient satisfies finite differences, the exact coupling derivative and
Euler's identity for homogeneous statistics."""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import adjoint as adj
from oracle import collision as col
from oracle import philox, vegas
from oracle.tasks import side_integrals


def _small(kind):
    if kind == "mb22":
        prob, f0 = W.c1_maxwell_2to2(n=8, neval=400, nitn=1)
    elif kind == "be23":
        prob, f0 = W.c3_cannibal_2to3(n=6, neval=300, nitn=1)
    else:
        prob, f0 = W.c4_multi_species(n=6, nmin=200, nmax=300, nitn=1)
    return prob, f0


def _maps(prob, seed=0):
    rng = np.random.default_rng(seed)
    maps = {}
    n = prob.grid.n
    for k, si in enumerate(side_integrals(prob)):
        nb = prob.processes[si.process].nbins
        for i in range(n):
            for term in (0, 1):
                w = rng.uniform(0.3, 2.0, size=(si.dim, nb))
                e = np.concatenate([np.zeros((si.dim, 1)), np.cumsum(w, axis=1)], axis=1)
                maps[(k * n + i) * 2 + term] = e / e[:, -1:]
    return maps


@pytest.mark.parametrize("kind", ["mb22", "be23", "multi"])
def test_torch_integrand_equals_numpy_integrand(kind):
    prob, f0 = _small(kind)
    t = 2.0 if kind == "multi" else 0.0
    q = col.grid_q(prob.grid)
    a = col.scale_factor(prob, t)
    m = col.masses(prob, t)
    dn = col.distributions(prob, f0, t)
    L = adj.spline_operator(q)
    f = torch.tensor(f0)
    mt = torch.tensor(m)
    dt_ = [adj.TorchDistribution(q, f[s], prob.species[s].stat, mt[s], a, prob.tail_points, L)
           for s in range(len(prob.species))]
    for k, si in enumerate(side_integrals(prob)):
        x = philox.uniforms(prob.seed, 3, 0, 0, 500, si.dim, "f64")
        y, jac, _ = vegas.apply_map(vegas.uniform_edges(si.dim, 50), x)
        for term in (0, 1):
            wn = col.integrand(prob, si, term, 2, f0[si.species][2], dn, m, a, y)
            wt = adj._integrand(prob, si, term, 2, f, dt_, mt, prob.processes[si.process].coupling, a, y, q)
            assert np.allclose(wt.numpy(), wn, rtol=1e-10, atol=1e-300)


@pytest.mark.parametrize("kind", ["mb22", "be23", "multi"])
def test_gradient_matches_central_differences(kind):
    prob, f0 = _small(kind)
    t = 2.0 if kind == "multi" else 0.0
    maps = _maps(prob)
    rng = np.random.default_rng(4)
    v = rng.normal(size=f0.shape)
    C, gf, gm, gl = adj.vjp(prob, f0, t, v, maps, 0)

    def L(f, m=None, lam=None):
        mm = torch.tensor(m if m is not None else [s.mass0 + s.mass1 * t for s in prob.species],
                          dtype=torch.float64)
        ll = torch.tensor(lam if lam is not None else [p.coupling for p in prob.processes], dtype=torch.float64)
        return float((adj.fixed_sample_C(prob, torch.tensor(f), mm, ll, t, maps, 0) * torch.tensor(v)).sum())

    h = 1e-4                      # relative step (smaller steps hit roundoff on tiny grid values)
    S, n = f0.shape
    for (s, j) in [(0, 0), (0, n // 2), (S - 1, n - 1), (S - 1, 1)]:
        if f0[s, j] < 1e-8 * f0.max():
            continue                  # a relative step cannot move L above roundoff there
        fp, fm = f0.copy(), f0.copy()
        fp[s, j] *= 1 + h
        fm[s, j] *= 1 - h
        fd = (L(fp) - L(fm)) / (2 * h * f0[s, j])
        assert abs(fd - gf[s, j]) <= 1e-4 * abs(gf[s, j]) + 1e-6 * np.max(np.abs(gf))
    m0 = np.array([s_.mass0 + s_.mass1 * t for s_ in prob.species])
    for s in range(S):
        if m0[s] == 0:
            continue
        mp, mm = m0.copy(), m0.copy()
        mp[s] *= 1 + h
        mm[s] *= 1 - h
        fd = (L(f0, m=mp) - L(f0, m=mm)) / (2 * h * m0[s])
        assert abs(fd - gm[s]) <= 1e-4 * abs(gm[s]) + 1e-12


def test_coupling_derivative_is_exact():
    """|M|^2 = lambda^2: dL/dlambda = 2 L / lambda (one process)."""
    prob, f0 = _small("mb22")
    maps = _maps(prob)
    v = np.ones_like(f0)
    C, gf, gm, gl = adj.vjp(prob, f0, 0.0, v, maps, 0)
    lam = prob.processes[0].coupling
    assert np.isclose(gl[0], 2.0 * np.sum(v * C) / lam, rtol=1e-12)


def test_euler_identity_for_maxwell_boltzmann():
    """MB 2 -> 2: gain and loss are products of two f values, each
    homogeneous of degree one in the grid values (spline linear; Eq. (13)
    tails shift by log c), so C~(c f) = c^2 C~(f) and sum_j f_j dC~/df_j = 2 C~."""
    prob, f0 = _small("mb22")
    maps = _maps(prob)
    rng = np.random.default_rng(5)
    v = rng.normal(size=f0.shape)
    C, gf, gm, gl = adj.vjp(prob, f0, 0.0, v, maps, 0)
    assert np.isclose(np.sum(f0 * gf), 2.0 * np.sum(v * C), rtol=1e-10)
