"""Distribution lookup: cubic spline inside the grid, Eq. (13) tails outside.

Test infrastructure (see ``oracle/__init__``).

Sec. 3B: between grid points f is a cubic spline in linear scale (linear in
both q and f); outside the grid, log(1/f + eta) = a + b E(p) with eta = +1
(BE), -1 (FD), 0 (MB) and E(p) = sqrt(p^2 + m^2), with (a, b) from linear fits
to the low and high ends of the grid separately.

Readings (the paper is silent on these):
  * the spline's end condition is not-a-knot (scipy's default);
  * each end fit is an ordinary least-squares line through the K =
    tail_points end grid points, in the variable E(q/a) with the current
    mass and scale factor;
  * a spline value below 0 is clamped to 0, and an FD value above 1 to 1;
  * a BE tail whose denominator exp(a + bE) - 1 is not positive gives f = 0.
"""
import numpy as np
from scipy.interpolate import CubicSpline

from workloads import STAT_BE, STAT_FD, STAT_MB

ETA = {STAT_MB: 0.0, STAT_BE: 1.0, STAT_FD: -1.0}


def line_fit(x, y):
    """Least-squares line y = a + b x; returns (a, b)."""
    xm, ym = np.mean(x), np.mean(y)
    b = np.sum((x - xm) * (y - ym)) / np.sum((x - xm) ** 2)
    return ym - b * xm, b


class Distribution:
    """f(q) of one species at one instant (grid values, mass, scale factor)."""

    def __init__(self, q, f, stat, mass, a=1.0, tail_points=4):
        self.q = np.asarray(q, dtype=np.float64)
        self.f = np.asarray(f, dtype=np.float64)
        self.stat = stat
        self.eta = ETA[stat]
        self.mass = float(mass)
        self.a = float(a)
        self.spline = CubicSpline(self.q, self.f, bc_type="not-a-knot")
        k = tail_points
        E = self.energy(self.q)
        y = np.log(1.0 / self.f + self.eta)
        self.tail_lo = line_fit(E[:k], y[:k])
        self.tail_hi = line_fit(E[-k:], y[-k:])

    def energy(self, q):
        p = np.asarray(q) / self.a
        return np.sqrt(p * p + self.mass * self.mass)

    def _tail(self, q, ab):
        x = ab[0] + ab[1] * self.energy(q)
        if self.eta == 1.0:
            den = np.expm1(x)
        else:
            den = np.exp(x) - self.eta
        with np.errstate(divide="ignore"):
            out = np.where(den > 0.0, 1.0 / np.where(den > 0.0, den, 1.0), 0.0)
        return out

    def __call__(self, q):
        q = np.asarray(q, dtype=np.float64)
        out = np.empty_like(q)
        inside = (q >= self.q[0]) & (q <= self.q[-1])
        lo = q < self.q[0]
        hi = q > self.q[-1]
        v = self.spline(q[inside])
        v = np.maximum(v, 0.0)
        if self.stat == STAT_FD:
            v = np.minimum(v, 1.0)
        out[inside] = v
        out[lo] = self._tail(q[lo], self.tail_lo)
        out[hi] = self._tail(q[hi], self.tail_hi)
        return out
