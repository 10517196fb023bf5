"""Monte Carlo collision integral C_a[f](p_i) -- the method's hot path.

Test infrastructure (see ``oracle/__init__``).

Per side integral and grid point the oracle estimates, separately for the
gain and the loss term (Sec. 2D), the single-position integral of Eq. (3)

    C^(k)(p) = 1/(2E) Int dPi |M|^2 Lambda,

parametrised as in Sec. 2D and App. A:
  * the observed leg sits on the z axis with physical momentum p = q_i / a;
  * each integrated leg has comoving (r, theta, phi) with r in
    [q_min, q_max], theta in [0, pi], phi in [0, 2 pi), Jacobian
    r^2 sin(theta) and a^-3 per leg (Sec. 3E), physical momentum r / a;
  * the conserved leg follows from 3-momentum conservation, Eq. (10) with the
    sign cases of App. A; its comoving momentum is |p_cons| a;
  * E_k = sqrt(|p_k|^2 + m_k^2); a sample with any E_k < E_cut has weight 0
    (App. A);
  * energy conservation uses the Gaussian of Eq. (11) with width sigma_E,
    or the fractional width w (E_in + E_out) / 2 of App. C (``width``);
  * the weight is Eq. (12) / App. A: prod r^2 sin(theta) over
    ((2 pi)^(3(n-1)-4) prod_{all n legs} 2E) times the Gaussian, times |M|^2
    and the gain or loss product; |M|^2 = coupling^2 P(s) with P a cubic in
    the invariant s of the initial state (the paper takes any callable of the
    momenta; its examples are all constant, P = 1);
  * gain = prod_{other side} f * prod_{observed side} (1 + eta f) and
    loss = prod_{observed side} f * prod_{other side} (1 + eta f), the f of
    the observed leg being the grid value f_a(q_i) (Sec. 2C, Eq. (5) and the
    explicit C_2 / C_3 products).
The unit cube is mapped to (r, theta, phi) by the VEGAS map followed by the
linear scaling, whose volume (q_max - q_min) pi 2 pi per leg multiplies the
weight.  C_a(p_i) = sum over side integrals of n_S^a (gain - loss) (Eq. (7)).
"""
from dataclasses import dataclass, field
from typing import Dict

import numpy as np

from workloads import PREC_FP32
from . import budget as obudget
from . import philox, stratified, vegas, width as owidth
from .spline import ETA, Distribution
from .tasks import SIDE_IN, side_integrals, task_id

TWO_PI = 2.0 * np.pi
CHUNK = 1 << 18


def grid_q(grid):
    """Comoving grid abscissae (Sec. 3A): log or linear, exact end points."""
    if grid.log_spaced:
        j = np.arange(grid.n)
        q = grid.q_min * (grid.q_max / grid.q_min) ** (j / (grid.n - 1))
    else:
        q = grid.q_min + (grid.q_max - grid.q_min) * np.arange(grid.n) / (grid.n - 1)
    q[0], q[-1] = grid.q_min, grid.q_max
    return q


def scale_factor(problem, t):
    """a(t): 1 without expansion, a0 (t/t0)^(1/2) under radiation domination (Sec. 3E)."""
    if problem.expansion is None:
        return 1.0
    return problem.expansion.a0 * np.sqrt(t / problem.expansion.t0)


def mass_of(species, t):
    """m(t) of one species (time-dependent mass, Sec. 3A): mass0 + mass1 t,
    or, when the species carries a knot table, the straight line between the
    two knots around t, and the end knot's mass beyond either end."""
    tab = species.mass_table
    if tab is None:
        return species.mass0 + species.mass1 * t
    if t <= tab[0][0]:
        return tab[0][1]
    for (ta, ma), (tb, mb) in zip(tab[:-1], tab[1:]):
        if t <= tb:
            return ma + (mb - ma) * ((t - ta) / (tb - ta))
    return tab[-1][1]


def masses(problem, t):
    """m_s(t) per species."""
    return np.array([mass_of(s, t) for s in problem.species])


def distributions(problem, f, t):
    q = grid_q(problem.grid)
    a = scale_factor(problem, t)
    m = masses(problem, t)
    return [Distribution(q, f[s], problem.species[s].stat, m[s], a, problem.tail_points)
            for s in range(len(problem.species))]


def kinematics(problem, si, i, m, a, y):
    """Momenta, energies and measure of the samples y (N, D) of a side integral.

    Returns (mom (n, N, 3) physical momenta, E (n, N), qcom (n, N) comoving
    magnitudes used for the f lookup, jac (N,) = prod over integrated legs of
    r^2 sin(theta) a^-3 times the volume of the linear scaling).
    """
    g = problem.grid
    n = si.n
    N = y.shape[0]
    q_i = grid_q(g)[i]
    mom = np.zeros((n, N, 3))
    qcom = np.zeros((n, N))
    jac = np.ones(N)
    mom[si.obs, :, 2] = q_i / a
    qcom[si.obs] = q_i
    for j, k in enumerate(si.integrated):
        r = g.q_min + (g.q_max - g.q_min) * y[:, 3 * j]
        th = np.pi * y[:, 3 * j + 1]
        ph = TWO_PI * y[:, 3 * j + 2]
        st = np.sin(th)
        mom[k, :, 0] = (r / a) * st * np.cos(ph)
        mom[k, :, 1] = (r / a) * st * np.sin(ph)
        mom[k, :, 2] = (r / a) * np.cos(th)
        qcom[k] = r
        jac *= r * r * st * (g.q_max - g.q_min) * np.pi * TWO_PI / a ** 3
    # Eq. (10) with the sign cases of App. A
    c = si.cons
    total = np.zeros((N, 3))
    for k in range(n):
        if k == c:
            continue
        total += mom[k] if si.is_in(k) else -mom[k]
    mom[c] = -total if si.is_in(c) else total
    qcom[c] = np.sqrt(np.sum(mom[c] ** 2, axis=1)) * a
    E = np.sqrt(np.sum(mom ** 2, axis=2) + (m[list(si.legs)] ** 2)[:, None])
    return mom, E, qcom, jac


def invariant_s(si, mom, E):
    """s = (sum of initial energies)^2 - |sum of initial momenta|^2 per sample."""
    Ein = sum(E[k] for k in range(si.n) if si.is_in(k))
    Pin = sum(mom[k] for k in range(si.n) if si.is_in(k))
    return Ein * Ein - np.sum(Pin * Pin, axis=-1)


def matrix_element_poly(proc, s):
    """|M|^2 / coupling^2 = c0 + c1 s + c2 s^2 + c3 s^3 (Horner)."""
    c = getattr(proc, "me_coef", (1.0, 0.0, 0.0, 0.0))
    return ((c[3] * s + c[2]) * s + c[1]) * s + c[0]


def integrand(problem, si, term, i, f_obs, dists, m, a, y, w_frac=None):
    """Integrand on the unit cube (before the VEGAS Jacobian), shape (N,);
    w_frac: the process's fractional width (default: its initial width)."""
    proc = problem.processes[si.process]
    n = si.n
    N = y.shape[0]
    mom, E, qcom, jac = kinematics(problem, si, i, m, a, y)
    cut = np.any(E < problem.e_cut, axis=0)
    dE = np.zeros(N)
    for k in range(n):
        dE += E[k] if si.is_in(k) else -E[k]
    sig = owidth.sigma(proc, proc.width if w_frac is None else w_frac, np.sum(E, axis=0))
    gauss = np.exp(-dE * dE / (2.0 * sig * sig)) / (sig * np.sqrt(2.0 * np.pi))
    # statistical factor, Eq. (5) with the observed-side products of Sec. 2C
    gain = np.ones(N)
    loss = np.ones(N)
    for k in range(n):
        sp = si.legs[k]
        if k == si.obs:
            fk = np.full(N, f_obs)
        else:
            fk = dists[sp](qcom[k])
        own = si.is_in(k) == (si.side == SIDE_IN)
        enh = 1.0 + ETA[problem.species[sp].stat] * fk
        if own:
            gain *= enh
            loss *= fk
        else:
            gain *= fk
            loss *= enh
    stat = gain if term == 0 else loss
    w = (proc.coupling ** 2) * matrix_element_poly(proc, invariant_s(si, mom, E)) * stat * jac * gauss / \
        (TWO_PI ** (3 * (n - 1) - 4) * np.prod(2.0 * E, axis=0))
    w[cut] = 0.0
    return w


@dataclass
class State:
    """Persistent VEGAS maps (one per task, reused across calls, Sec. 3D),
    the counter of collision evaluations (part of the sample stream) and the
    fractional Gaussian width of each process (App. C) with the relative
    error that set it."""
    maps: Dict[int, np.ndarray] = field(default_factory=dict)
    call: int = 0
    widths: Dict[int, float] = field(default_factory=dict)
    width_rel: Dict[int, float] = field(default_factory=dict)
    strata: Dict[int, np.ndarray] = field(default_factory=dict)
    budgets: Dict[int, int] = field(default_factory=dict)     # variance-driven budgets of the next sweep


def task_budget(proc, i):
    """Samples per iteration of a task (stratified: whole items of 8)."""
    N = proc.neval_per_point[i] if proc.neval_per_point is not None else proc.neval
    if getattr(proc, "strat", 0):
        N = stratified.CHUNK_ITEMS * (N // stratified.CHUNK_ITEMS)
    return N


def evaluate_task(problem, si_index, si, i, term, f, t, edges, call, mode="f64", dists=None, w_frac=None,
                  strata=None, N=None):
    """Run the nitn VEGAS iterations of one task.

    Returns (mean, err, edges_after, per-iteration list of (mean, var),
    strata_after); strata is the stratified allocation (items per hypercube)
    or None without stratification.
    """
    proc = problem.processes[si.process]
    if dists is None:
        dists = distributions(problem, f, t)
    a = scale_factor(problem, t)
    m = masses(problem, t)
    f_obs = f[si.species][i]
    D = si.dim
    N = task_budget(proc, i) if N is None else int(N)
    tid = task_id(si_index, i, term, problem.grid.n)
    strat = bool(getattr(proc, "strat", 0))
    if strat:
        M, H, J = stratified.shape(N, D, proc.strat_max_hcubes)
        alloc = strata if strata is not None else stratified.uniform_allocation(J, H)
    iters = []
    for it in range(proc.nitn):
        sw = 0.0
        sw2 = 0.0
        d = np.zeros((D, proc.nbins))
        if strat:
            item_h = np.repeat(np.arange(H), alloc)
            S1 = np.zeros(H)
            S2 = np.zeros(H)
        for s0 in range(0, N, CHUNK):
            ns = min(CHUNK, N - s0)
            x = philox.uniforms(problem.seed, tid, it, call, ns, D, mode, first_sample=s0)
            if strat:
                h = item_h[np.arange(s0, s0 + ns) // stratified.CHUNK_ITEMS]
                x = (stratified.digits(h, M, D) + x) / M
            y, jac, bins = vegas.apply_map(edges, x)
            w = integrand(problem, si, term, i, f_obs, dists, m, a, y, w_frac) * jac
            if strat:
                np.add.at(S1, h, w)
                np.add.at(S2, h, w * w)
                w2m = w * w / alloc[h]
                d += np.stack([np.bincount(bins[:, k], weights=w2m, minlength=proc.nbins) for k in range(D)])
            else:
                sw += np.sum(w)
                sw2 += np.sum(w * w)
                d += vegas.training_data(bins, w, proc.nbins)
        if strat:
            mean_it, var_it, s2 = stratified.estimate(S1, S2, alloc)
            iters.append((mean_it, var_it))
            alloc = stratified.allocate(s2, J, proc.strat_beta)
        else:
            iters.append(vegas.iteration_estimate(sw, sw2, N))
        edges = vegas.refine(edges, d, proc.alpha)
    mean, err = vegas.combine([v[0] for v in iters], [v[1] for v in iters])
    return mean, err, edges, iters, (alloc if strat else None)


def collision(problem, f, t, state, mode="f64", points=None):
    """C_a(p_i) and its MC standard error for every species and grid point.

    ``points`` restricts the evaluation to some grid points (others stay 0);
    the maps of evaluated tasks are updated in ``state``.  Returns
    (C, err, detail) with detail[task_id] = (mean, err) per gain/loss task.
    """
    f = np.asarray(f, dtype=np.float64)
    S, n = f.shape
    C = np.zeros((S, n))
    var = np.zeros((S, n))
    detail = {}
    pts = range(n) if points is None else points
    dists = distributions(problem, f, t)
    widths = {p: state.widths.get(p, proc.width) for p, proc in enumerate(problem.processes)}
    per_process = {p: ([], []) for p in range(len(problem.processes))}
    used = {p: [] for p in range(len(problem.processes))}          # (task id, budget, mean, err)
    for k, si in enumerate(side_integrals(problem)):
        nb = problem.processes[si.process].nbins
        for i in pts:
            res = []
            for term in (0, 1):
                tid = task_id(k, i, term, n)
                edges = state.maps.get(tid)
                if edges is None:
                    edges = vegas.uniform_edges(si.dim, nb)
                N = state.budgets.get(tid, task_budget(problem.processes[si.process], i))
                mean, err, edges, _, alloc = evaluate_task(problem, k, si, i, term, f, t, edges, state.call,
                                                           mode, dists, widths[si.process], state.strata.get(tid),
                                                           N)
                used[si.process].append((tid, N, mean, err))
                state.maps[tid] = edges
                if alloc is not None:
                    state.strata[tid] = alloc
                detail[tid] = (mean, err)
                res.append((mean, err))
                per_process[si.process][0].append(mean)
                per_process[si.process][1].append(err)
            (Ig, eg), (Il, el) = res
            C[si.species, i] += si.mult * (Ig - Il)
            var[si.species, i] += si.mult ** 2 * (eg * eg + el * el)
    for p, proc in enumerate(problem.processes):
        rel = owidth.relative_error(*per_process[p])
        state.widths[p] = owidth.adapt(widths[p], rel, proc)
        state.width_rel[p] = rel
        if getattr(proc, "budget", 0) and used[p]:
            # variance-driven budgets of the next sweep; the pool is the
            # process's tasks evaluated here, its total their configured budgets
            tids, Ns, means, errs = (np.array(c) for c in zip(*used[p]))
            total = float(sum(task_budget(proc, (tid // 2) % n) for tid in tids))
            nxt = obudget.next_budgets(Ns, means, errs, total, proc.neval_min, proc.neval_max)
            state.budgets.update({int(tid): int(b) for tid, b in zip(tids, nxt)})
    state.call += 1
    return C, np.sqrt(var), detail


def uniform_mode(precision):
    return "f32" if precision == PREC_FP32 else "f64"
