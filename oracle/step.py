"""Log-space time integration with adaptive dt (Sec. 3C).

Test infrastructure (see ``oracle/__init__``).

Euler, Eq. (14):  log f(t+dt) = log f(t) + dt C[f]/f.
Heun, Eq. (15):   f* = exp(log f + dt k1/f), k2 = C[f*] at t + dt,
                  log f(t+dt) = log f(t) + dt/2 (k1/f + k2/f*).
Adaptive step, Eq. (16): max_p |dt C/f| < eps.  Reading: the step used is
dt = min(dt_requested, eps / max_p |k1/f|), taken from k1 and used by both
stages of Heun; k2 is evaluated at time t + dt (masses and a(t) there).
"""
import numpy as np

from .collision import collision


def limit_dt(dt, C, f, eps):
    rate = float(np.max(np.abs(C / f)))
    if rate > 0.0:
        return min(dt, eps / rate)
    return dt


def euler(rhs, logf, t, dt, eps):
    """Eq. (14) with the step bound of Eq. (16); rhs(f, t) -> C.
    Returns (logf_new, t_new, dt_used, C)."""
    f = np.exp(logf)
    C = rhs(f, t)
    dt = limit_dt(dt, C, f, eps)
    return logf + dt * C / f, t + dt, dt, C


def heun(rhs, logf, t, dt, eps):
    """Eq. (15) with the step bound of Eq. (16) taken from k1.
    Returns (logf_new, t_new, dt_used, k1, k2)."""
    f = np.exp(logf)
    k1 = rhs(f, t)
    dt = limit_dt(dt, k1, f, eps)
    f_star = np.exp(logf + dt * k1 / f)
    k2 = rhs(f_star, t + dt)
    return logf + 0.5 * dt * (k1 / f + k2 / f_star), t + dt, dt, k1, k2


def collision_rhs(problem, state, mode="f64"):
    """rhs(f, t) = C[f] from the Monte Carlo collision integral."""
    return lambda f, t: collision(problem, f, t, state, mode)[0]


def euler_step(problem, logf, t, dt, state, mode="f64"):
    return euler(collision_rhs(problem, state, mode), logf, t, dt, problem.eps_dt)


def heun_step(problem, logf, t, dt, state, mode="f64"):
    return heun(collision_rhs(problem, state, mode), logf, t, dt, problem.eps_dt)
