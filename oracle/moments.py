"""Number and energy densities of each species (conservation diagnostics of
the thermalisation runs, Sec. 5C / Fig. 3).

Test infrastructure (see ``oracle/__init__``).

Reading (the paper plots the relative change of the total number and energy
without stating the quadrature): for species s at time t,

    n_s   = 1 / (2 pi^2 a^3) Int_{q_min}^{q_max} q^2 f_s(q) dq,
    rho_s = 1 / (2 pi^2 a^3) Int_{q_min}^{q_max} q^2 E_s(q / a) f_s(q) dq,

one internal degree of freedom, physical momentum p = q / a, f the
not-a-knot cubic spline of the grid values (not clamped; the Eq. (13)
tails outside the grid are not included), each grid interval integrated by
4-point Gauss-Legendre (exact for n, whose integrand is a polynomial of
degree 5 in q).
"""
import numpy as np
from scipy.interpolate import CubicSpline

from .collision import grid_q, masses, scale_factor

GL_NODES = 4


def moments(problem, f, t):
    """(n[S], rho[S]) of the grid values f (S, n) at time t."""
    q = grid_q(problem.grid)
    a = scale_factor(problem, t)
    m = masses(problem, t)
    x, w = np.polynomial.legendre.leggauss(GL_NODES)
    lo, hi = q[:-1], q[1:]
    half = 0.5 * (hi - lo)
    qq = (0.5 * (hi + lo))[:, None] + half[:, None] * x[None, :]       # (n-1, 4)
    ww = half[:, None] * w[None, :]
    pref = 1.0 / (2.0 * np.pi ** 2 * a ** 3)
    n_out, r_out = [], []
    for s in range(len(problem.species)):
        sp = CubicSpline(q, np.asarray(f[s], dtype=np.float64), bc_type="not-a-knot")
        fv = sp(qq)
        E = np.sqrt((qq / a) ** 2 + m[s] ** 2)
        n_out.append(pref * np.sum(ww * qq ** 2 * fv))
        r_out.append(pref * np.sum(ww * qq ** 2 * E * fv))
    return np.array(n_out), np.array(r_out)
