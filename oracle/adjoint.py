"""Differentiable fixed-sample collision integral (the adjoint's oracle).

Test infrastructure (see ``oracle/__init__``).  The paper has no gradients;
this module defines what the library's adjoint differentiates and computes
its gradient by reverse-mode automatic differentiation (PyTorch, FP64 CPU).

C~_a(p_i) is the collision integral of Eq. (7) estimated with ONE VEGAS
iteration per task on a given, fixed map and a fixed sample stream (Philox
iteration index VJP_ITERATION, evaluation counter `call`), i.e. with common
random numbers: a deterministic, piecewise smooth function of the grid values
f_j of every species, of the masses m_s and of the couplings.  Everything
the samples depend on (uniforms, map, Jacobian) is independent of those
parameters; the integrand is the restatement of ``collision.integrand`` with
the spline built as a linear map of the grid values (scipy's not-a-knot
spline applied to unit vectors) so that it is differentiable, and the tails
of Eq. (13) fitted with the least-squares formula in torch.
"""
import numpy as np
import torch
from scipy.interpolate import CubicSpline

from . import philox, vegas, width as owidth
from .collision import TWO_PI, grid_q, masses, scale_factor, task_budget
from .spline import ETA
from .tasks import SIDE_IN, side_integrals, task_id

VJP_ITERATION = 0xFFFF


def spline_operator(q):
    """L with coef = L @ f: the not-a-knot spline's interval coefficients
    (c0..c3 of c0 + c1 t + c2 t^2 + c3 t^3, t = x - q_j) are linear in f."""
    n = len(q)
    L = np.zeros((n - 1, 4, n))
    for j in range(n):
        e = np.zeros(n)
        e[j] = 1.0
        c = CubicSpline(q, e, bc_type="not-a-knot").c      # (4, n-1), highest power first
        L[:, :, j] = c[::-1].T
    return torch.tensor(L)


class TorchDistribution:
    """f(q) of one species as a differentiable function of (f_grid, mass)."""

    def __init__(self, q, f, stat, mass, a, tail_points, L):
        self.q = q
        self.qt = torch.tensor(q)
        self.f = f
        self.stat = stat
        self.eta = ETA[stat]
        self.mass = mass
        self.a = a
        self.coef = torch.einsum("jkn,n->jk", L, f)              # (n-1, 4)
        k = tail_points
        E = torch.sqrt((self.qt / a) ** 2 + mass ** 2)
        y = torch.log(1.0 / f + self.eta)
        self.tail_lo = self._fit(E[:k], y[:k])
        self.tail_hi = self._fit(E[-k:], y[-k:])

    @staticmethod
    def _fit(x, y):
        xm, ym = x.mean(), y.mean()
        b = ((x - xm) * (y - ym)).sum() / ((x - xm) ** 2).sum()
        return ym - b * xm, b

    def __call__(self, qv):
        """qv: numpy comoving momenta (independent of the parameters)."""
        out = torch.zeros(len(qv), dtype=torch.float64)
        inside = (qv >= self.q[0]) & (qv <= self.q[-1])
        if inside.any():
            qi = qv[inside]
            j = np.clip(np.searchsorted(self.q, qi, side="right") - 1, 0, len(self.q) - 2)
            t = torch.tensor(qi - self.q[j])
            c = self.coef[j]
            v = ((c[:, 3] * t + c[:, 2]) * t + c[:, 1]) * t + c[:, 0]
            v = torch.clamp(v, min=0.0)
            if self.eta == -1.0:
                v = torch.clamp(v, max=1.0)
            out = out.index_put((torch.tensor(np.flatnonzero(inside)),), v)
        for mask, (a0, b) in ((qv < self.q[0], self.tail_lo), (qv > self.q[-1], self.tail_hi)):
            if mask.any():
                E = torch.sqrt(torch.tensor(qv[mask] / self.a) ** 2 + self.mass ** 2)
                x = a0 + b * E
                den = torch.expm1(x) if self.eta == 1.0 else torch.exp(x) - self.eta
                v = torch.where(den > 0, 1.0 / torch.where(den > 0, den, torch.ones_like(den)),
                                torch.zeros_like(den))
                if self.eta == -1.0:
                    v = torch.clamp(v, max=1.0)
                out = out.index_put((torch.tensor(np.flatnonzero(mask)),), v)
        return out


def fixed_sample_C(problem, f, masses, couplings, t, maps, call, mode="f64", widths=None):
    """C~ (n_species, n_grid) as a torch function of f (S, n), masses (S,)
    and couplings (P,); maps[task] = edges (D, nb+1) numpy; widths[p]: the
    fractional Gaussian width of process p (default: its initial width)."""
    g = problem.grid
    q = grid_q(g)
    a = scale_factor(problem, t)
    L = spline_operator(q)
    S, n = f.shape
    dists = [TorchDistribution(q, f[s], problem.species[s].stat, masses[s], a, problem.tail_points, L)
             for s in range(S)]
    rows = [[torch.zeros((), dtype=torch.float64) for _ in range(n)] for _ in range(S)]
    for k, si in enumerate(side_integrals(problem)):
        proc = problem.processes[si.process]
        D = si.dim
        for i in range(n):
            for term in (0, 1):
                tid = task_id(k, i, term, n)
                N = task_budget(proc, i)
                x = philox.uniforms(problem.seed, tid, VJP_ITERATION, call, N, D, mode)
                y, jac, _ = vegas.apply_map(maps[tid], x)
                wf = proc.width if widths is None else widths[si.process]
                w = _integrand(problem, si, term, i, f, dists, masses, couplings[si.process], a, y, q, wf) * \
                    torch.tensor(jac)
                sign = 1.0 if term == 0 else -1.0
                rows[si.species][i] = rows[si.species][i] + si.mult * sign * w.mean()
    return torch.stack([torch.stack(r) for r in rows])


def _integrand(problem, si, term, i, f, dists, masses, coupling, a, y, q, w_frac=None):
    proc = problem.processes[si.process]
    gr = problem.grid
    n = si.n
    N = y.shape[0]
    mom = {}
    qcom = {}
    jac = np.ones(N)
    mom[si.obs] = np.zeros((N, 3))
    mom[si.obs][:, 2] = q[i] / a
    for j, k in enumerate(si.integrated):
        r = gr.q_min + (gr.q_max - gr.q_min) * y[:, 3 * j]
        th = np.pi * y[:, 3 * j + 1]
        ph = TWO_PI * y[:, 3 * j + 2]
        st = np.sin(th)
        mom[k] = np.stack([(r / a) * st * np.cos(ph), (r / a) * st * np.sin(ph), (r / a) * np.cos(th)], axis=1)
        qcom[k] = r
        jac = jac * r * r * st * (gr.q_max - gr.q_min) * np.pi * TWO_PI / a ** 3
    c = si.cons
    total = np.zeros((N, 3))
    for k in range(n):
        if k != c:
            total = total + (mom[k] if si.is_in(k) else -mom[k])
    mom[c] = -total if si.is_in(c) else total
    qcom[c] = np.sqrt(np.sum(mom[c] ** 2, axis=1)) * a
    E = {}
    for k in range(n):
        p2 = torch.tensor(np.sum(mom[k] ** 2, axis=1))
        E[k] = torch.sqrt(p2 + masses[si.legs[k]] ** 2)
    cut = torch.zeros(N, dtype=torch.bool)
    for k in range(n):
        cut = cut | (E[k] < problem.e_cut)
    dE = sum(E[k] if si.is_in(k) else -E[k] for k in range(n))
    sig = owidth.sigma(proc, proc.width if w_frac is None else w_frac, sum(E[k] for k in range(n)))
    gauss = torch.exp(-dE * dE / (2.0 * sig * sig)) / (sig * np.sqrt(2.0 * np.pi))
    gain = torch.ones(N, dtype=torch.float64)
    loss = torch.ones(N, dtype=torch.float64)
    for k in range(n):
        sp = si.legs[k]
        fk = f[sp, i].expand(N) if k == si.obs else dists[sp](qcom[k])
        own = si.is_in(k) == (si.side == SIDE_IN)
        enh = 1.0 + ETA[problem.species[sp].stat] * fk
        if own:
            gain = gain * enh
            loss = loss * fk
        else:
            gain = gain * fk
            loss = loss * enh
    stat = gain if term == 0 else loss
    prodE = torch.ones(N, dtype=torch.float64)
    for k in range(n):
        prodE = prodE * 2.0 * E[k]
    Ein = sum(E[k] for k in range(n) if si.is_in(k))
    Pin = sum(mom[k] for k in range(n) if si.is_in(k))
    s_inv = Ein * Ein - torch.tensor(np.sum(Pin * Pin, axis=1))
    c = getattr(proc, "me_coef", (1.0, 0.0, 0.0, 0.0))
    me = ((c[3] * s_inv + c[2]) * s_inv + c[1]) * s_inv + c[0]
    w = coupling ** 2 * me * stat * torch.tensor(jac) * gauss / (TWO_PI ** (3 * (n - 1) - 4) * prodE)
    return torch.where(cut, torch.zeros_like(w), w)


def vjp(problem, f0, t, v, maps, call, mode="f64", widths=None):
    """(C~, dL/df, dL/dm, dL/dcoupling) for L = sum(v * C~)."""
    f = torch.tensor(np.asarray(f0, dtype=np.float64), requires_grad=True)
    m = torch.tensor(masses(problem, t), dtype=torch.float64, requires_grad=True)
    lam = torch.tensor([p.coupling for p in problem.processes], dtype=torch.float64, requires_grad=True)
    C = fixed_sample_C(problem, f, m, lam, t, maps, call, mode, widths)
    Lv = (C * torch.tensor(np.asarray(v, dtype=np.float64))).sum()
    gf, gm, gl = torch.autograd.grad(Lv, [f, m, lam], allow_unused=True)
    z = lambda g, like: g if g is not None else torch.zeros_like(like)
    return C.detach().numpy(), z(gf, f).numpy(), z(gm, m).numpy(), z(gl, lam).numpy()


def jvp(problem, f0, t, u, maps, call, mode="f64", widths=None):
    """(C~, J u) with J = dC~/df at fixed masses and couplings: the
    directional derivative of ``fixed_sample_C`` along u (forward mode, by
    torch's double-backward construction)."""
    m = torch.tensor(masses(problem, t), dtype=torch.float64)
    lam = torch.tensor([p.coupling for p in problem.processes], dtype=torch.float64)
    f = torch.tensor(np.asarray(f0, dtype=np.float64))
    ut = torch.tensor(np.asarray(u, dtype=np.float64))
    C, Ju = torch.autograd.functional.jvp(lambda ff: fixed_sample_C(problem, ff, m, lam, t, maps, call, mode,
                                                                    widths),
                                          (f,), (ut,))
    return C.detach().numpy(), Ju.detach().numpy()
