"""Implicit (backward) Euler in log space on the fixed-sample integral.

Test infrastructure (see ``oracle/__init__``).

The paper integrates log f explicitly (Eq. (14), (15)); its backward-Euler
counterpart takes g = log f(t + dt) as the root of

    R(g) = g - g_n - dt Q(g),    Q(g) = C~(e^g) / e^g,

with C~ evaluated at t + dt.  The oracle solves it with Newton's method on
the dense Jacobian  J_R = I - dt dQ/dg,  dQ/dg = diag(1/f) J diag(f) -
diag(C~/f), J = dC~/df from automatic differentiation of
``adjoint.fixed_sample_C`` (one column per unknown), and a direct linear
solve: no Krylov method, no damping unless the full step fails to reduce
||R||.  Small problems only.
"""
import numpy as np
import torch

from . import adjoint
from .collision import masses


def newton(residual, jacobian, g0, tol, max_iter=50):
    """Root of residual(g) by Newton's method with step halving on ||R||_2.
    Returns (g, iterations, ||R||_inf)."""
    g = np.array(g0, dtype=np.float64)
    r = residual(g)
    it = 0
    while np.max(np.abs(r)) > tol and it < max_iter:
        d = np.linalg.solve(jacobian(g), -r)
        lam = 1.0
        while True:
            gt = g + lam * d
            rt = residual(gt)
            if np.linalg.norm(rt) <= (1.0 - 1e-4 * lam) * np.linalg.norm(r) or lam < 1e-3:
                break
            lam *= 0.5
        g, r = gt, rt
        it += 1
    return g, it, float(np.max(np.abs(r)))


def implicit_euler(Q, dQ, g_n, dt, tol, max_iter=50):
    """Backward Euler g = g_n + dt Q(g) for a log-space right-hand side Q
    with Jacobian dQ (both callables of g)."""
    g_n = np.asarray(g_n, dtype=np.float64)
    res = lambda g: g - g_n - dt * Q(g)
    jac = lambda g: np.eye(g.size) - dt * dQ(g)
    return newton(res, jac, g_n, tol, max_iter)


def collision_step(problem, logf, t, dt, maps, call, tol=1e-12, mode="f64"):
    """One backward-Euler step of the fixed-sample collision integral at
    t + dt, maps and evaluation counter given.  Returns (logf_new,
    iterations, ||R||_inf)."""
    shape = np.shape(logf)
    t1 = t + dt
    m = torch.tensor(masses(problem, t1), dtype=torch.float64)
    lam = torch.tensor([p.coupling for p in problem.processes], dtype=torch.float64)

    def C_of(g):
        f = torch.exp(g.reshape(shape))
        return adjoint.fixed_sample_C(problem, f, m, lam, t1, maps, call, mode).reshape(-1)

    def Q(g):
        gt = torch.tensor(g)
        with torch.no_grad():
            return (C_of(gt) / torch.exp(gt)).numpy()

    def dQ(g):
        gt = torch.tensor(g)
        return torch.autograd.functional.jacobian(lambda x: C_of(x) / torch.exp(x), gt).numpy()

    g, it, rinf = implicit_euler(Q, dQ, np.asarray(logf, dtype=np.float64).reshape(-1), dt, tol)
    return g.reshape(shape), it, rinf
