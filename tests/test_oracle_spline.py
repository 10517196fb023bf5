"""Pins of the oracle's distribution lookup (Sec. 3B, Eq. (13))."""
import numpy as np
import pytest

from oracle.spline import Distribution, line_fit
from workloads import STAT_BE, STAT_FD, STAT_MB


def _grid(n=24, lo=0.05, hi=12.0):
    return np.geomspace(lo, hi, n)


def test_reproduces_cubics_exactly():
    """Not-a-knot splines reproduce any cubic (the knot conditions are then
    satisfied by the cubic itself), on a non-uniform grid."""
    q = _grid()
    poly = lambda x: 0.3 - 0.2 * x + 0.05 * x ** 2 + 0.004 * x ** 3
    d = Distribution(q, poly(q) + 2.0, STAT_MB, 1.0)
    x = np.linspace(q[0], q[-1], 777)
    assert np.allclose(d(x), poly(x) + 2.0, rtol=1e-12, atol=1e-12)


def test_not_a_knot_condition():
    """The third derivative is continuous across the second and the
    second-to-last knots (the definition of the not-a-knot end condition)."""
    q = _grid()
    f = 1.0 / (1.0 + np.exp(q - 3.0)) + 0.1
    d = Distribution(q, f, STAT_MB, 0.0)
    s3 = d.spline.c[0] * 6.0          # third derivative per interval
    assert np.isclose(s3[0], s3[1], rtol=1e-9)
    assert np.isclose(s3[-1], s3[-2], rtol=1e-9)
    assert np.allclose(d(q), f, rtol=1e-14)


@pytest.mark.parametrize("stat,eta", [(STAT_MB, 0.0), (STAT_BE, 1.0), (STAT_FD, -1.0)])
@pytest.mark.parametrize("mass,a", [(0.0, 1.0), (1.0, 1.0), (0.5, 2.0)])
def test_tails_exact_for_equilibrium(stat, eta, mass, a):
    """Eq. (13) is exact for equilibrium: f = 1/(exp((E - mu)/T) - eta) is
    recovered outside the grid, with E the physical energy at p = q/a."""
    T, mu = 0.8, -0.3
    q = _grid()
    E = lambda x: np.sqrt((x / a) ** 2 + mass ** 2)
    feq = lambda x: 1.0 / (np.exp((E(x) - mu) / T) - eta)
    d = Distribution(q, feq(q), stat, mass, a=a, tail_points=4)
    xo = np.concatenate([np.geomspace(1e-4, q[0] * 0.999, 7), np.geomspace(q[-1] * 1.001, 60.0, 7)])
    assert np.allclose(d(xo), feq(xo), rtol=1e-9)
    assert np.isclose(d.tail_hi[1], 1.0 / T) and np.isclose(d.tail_lo[0], -mu / T)


def test_tail_fit_is_least_squares():
    """The end fit minimises the squared residual: perturbing (a, b) raises it."""
    rng = np.random.default_rng(0)
    x = rng.uniform(1, 3, 4)
    y = 0.5 + 2.0 * x + rng.normal(0, 0.1, 4)
    a, b = line_fit(x, y)
    res = lambda a_, b_: np.sum((y - a_ - b_ * x) ** 2)
    r0 = res(a, b)
    for da, db in ((1e-3, 0), (-1e-3, 0), (0, 1e-3), (0, -1e-3)):
        assert res(a + da, b + db) > r0
    ref = np.polyfit(x, y, 1)
    assert np.allclose([b, a], ref)


def test_clamping():
    q = _grid(12, 0.1, 5.0)
    f = np.where(q < 1.0, 1e-3, 0.9)    # a step makes the spline overshoot
    d = Distribution(q, f, STAT_FD, 0.0)
    x = np.linspace(q[0], q[-1], 2001)
    v = d(x)
    assert v.min() >= 0.0 and v.max() <= 1.0
