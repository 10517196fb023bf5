"""Pins of the forward-mode tangent of the fixed-sample integral and of the
backward-Euler oracle: central differences, the adjoint identity, Euler's
homogeneity identity, closed-form backward-Euler solutions (linear and
Lambert-W), and the O(dt^2) distance to the explicit step."""
import numpy as np
import pytest
import torch
from scipy.special import lambertw

import workloads as W
from oracle import adjoint as adj
from oracle import implicit as imp
from oracle.tasks import side_integrals


def _small(kind):
    if kind == "mb22":
        return W.c1_maxwell_2to2(n=8, neval=400, nitn=1)
    if kind == "be23":
        return W.c3_cannibal_2to3(n=6, neval=300, nitn=1)
    return W.c4_multi_species(n=6, nmin=200, nmax=300, nitn=1)


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


def _C(prob, f, t, maps):
    m = torch.tensor([s.mass0 + s.mass1 * t for s in prob.species], dtype=torch.float64)
    lam = torch.tensor([p.coupling for p in prob.processes], dtype=torch.float64)
    with torch.no_grad():
        return adj.fixed_sample_C(prob, torch.tensor(f), m, lam, t, maps, 0).numpy()


@pytest.mark.parametrize("kind", ["mb22", "be23", "multi"])
def test_jvp_matches_central_differences(kind):
    prob, f0 = _small(kind)
    t = 2.0 if kind == "multi" else 0.0
    maps = _maps(prob)
    rng = np.random.default_rng(11)
    u = f0 * rng.normal(size=f0.shape)          # relative perturbation of every grid value
    C, Ju = adj.jvp(prob, f0, t, u, maps, 0)
    h = 1e-5
    fd = (_C(prob, f0 + h * u, t, maps) - _C(prob, f0 - h * u, t, maps)) / (2 * h)
    assert np.max(np.abs(fd - Ju)) <= 1e-5 * np.max(np.abs(Ju))
    assert np.allclose(C, _C(prob, f0, t, maps), rtol=1e-13, atol=0)


@pytest.mark.parametrize("kind", ["mb22", "multi"])
def test_jvp_is_the_transpose_of_the_vjp(kind):
    """<v, J u> = <J^T v, u> (the reverse-mode gradient)."""
    prob, f0 = _small(kind)
    t = 2.0 if kind == "multi" else 0.0
    maps = _maps(prob)
    rng = np.random.default_rng(12)
    u = rng.normal(size=f0.shape)
    v = rng.normal(size=f0.shape)
    _, Ju = adj.jvp(prob, f0, t, u, maps, 0)
    _, gf, _, _ = adj.vjp(prob, f0, t, v, maps, 0)
    lhs, rhs = np.sum(v * Ju), np.sum(gf * u)
    assert abs(lhs - rhs) <= 1e-10 * (np.sum(np.abs(v * Ju)) + 1e-300)


def test_jvp_euler_identity_for_maxwell_boltzmann():
    """MB 2 -> 2 is homogeneous of degree two in f: J f = 2 C~."""
    prob, f0 = _small("mb22")
    maps = _maps(prob)
    C, Jf = adj.jvp(prob, f0, 0.0, f0, maps, 0)
    assert np.allclose(Jf, 2.0 * C, rtol=1e-10, atol=1e-12 * np.max(np.abs(C)))


def test_newton_backward_euler_linear_closed_form():
    """Q(g) = -k (g - c): g = (g_n + dt k c) / (1 + dt k)."""
    rng = np.random.default_rng(1)
    k = rng.uniform(0.1, 50.0, size=7)
    c = rng.normal(size=7)
    gn = rng.normal(size=7)
    dt = 0.3
    g, it, rinf = imp.implicit_euler(lambda g: -k * (g - c), lambda g: np.diag(-k), gn, dt, 1e-14)
    assert np.allclose(g, (gn + dt * k * c) / (1 + dt * k), rtol=1e-13, atol=1e-14)
    assert it == 1                      # linear: one Newton step


def test_newton_backward_euler_relaxation_lambert_w():
    """Relaxation df/dt = -k (f - f_eq) in log space, Q(g) = -k (1 - f_eq e^-g):
    the backward-Euler root is g = B + W(A e^-B), A = dt k f_eq, B = g_n - dt k."""
    rng = np.random.default_rng(2)
    k = rng.uniform(0.5, 20.0, size=5)
    feq = rng.uniform(0.01, 3.0, size=5)
    gn = np.log(rng.uniform(0.01, 3.0, size=5))
    dt = 0.7
    Q = lambda g: -k * (1.0 - feq * np.exp(-g))
    dQ = lambda g: np.diag(-k * feq * np.exp(-g))
    g, it, rinf = imp.implicit_euler(Q, dQ, gn, dt, 1e-14)
    A, B = dt * k * feq, gn - dt * k
    want = B + np.real(lambertw(A * np.exp(-B)))
    assert np.allclose(g, want, rtol=1e-12, atol=1e-12)
    assert rinf <= 1e-14


def test_collision_backward_euler_converges_and_is_first_order():
    """On the fixed-sample integral: the residual reaches the tolerance and
    the distance to the explicit step with the same samples shrinks like dt^2."""
    prob, f0 = _small("mb22")
    maps = _maps(prob)
    g0 = np.log(f0)
    Q0 = _C(prob, f0, 0.0, maps) / f0
    rate = np.max(np.abs(Q0))
    d = []
    for dt in (0.05 / rate, 0.025 / rate):
        g, it, rinf = imp.collision_step(prob, g0, 0.0, dt, maps, 0, tol=1e-12)
        assert rinf <= 1e-12 and it <= 8
        d.append(np.max(np.abs(g - (g0 + dt * Q0))))
    assert 3.0 < d[0] / d[1] < 5.0
