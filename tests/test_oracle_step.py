"""Pins of the oracle's log-space Euler / Heun stepping (Sec. 3C)."""
import numpy as np

from oracle import step


def _linear(kappa, feq):
    return lambda f, t: -kappa * (f - feq)


def _solve(method, dt, T=1.0):
    kappa, feq = 1.3, np.array([0.2, 0.5, 1.0])
    logf = np.log(np.array([0.9, 0.1, 2.0]))
    t = 0.0
    n = int(round(T / dt))
    for _ in range(n):
        out = method(_linear(kappa, feq), logf, t, dt, eps=10.0)
        logf, t = out[0], out[1]
    exact = feq + (np.array([0.9, 0.1, 2.0]) - feq) * np.exp(-kappa * T)
    return np.max(np.abs(np.exp(logf) - exact))


def test_euler_first_order():
    e1, e2 = _solve(step.euler, 0.02), _solve(step.euler, 0.01)
    assert 1.8 < e1 / e2 < 2.2


def test_heun_second_order():
    e1, e2 = _solve(step.heun, 0.04), _solve(step.heun, 0.02)
    assert 3.6 < e1 / e2 < 4.4
    assert e2 < 0.05 * _solve(step.euler, 0.02)


def test_adaptive_step_bound():
    """Eq. (16): the step is cut so that max |dt C/f| = eps."""
    f = np.array([0.5, 0.01])
    rhs = lambda f_, t: np.array([0.1, -0.2])
    logf, t, dt, C = step.euler(rhs, np.log(f), 0.0, 1.0, 0.3)
    assert np.isclose(dt, 0.3 / 20.0)
    assert np.isclose(np.max(np.abs(dt * C / f)), 0.3)
    logf, t, dt, k1, k2 = step.heun(rhs, np.log(f), 0.0, 0.001, 0.3)
    assert dt == 0.001 and t == 0.001
