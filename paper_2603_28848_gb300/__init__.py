"""GB300 collision-integral library: Python binding of libbest.so.

Every step of the Monte Carlo collision integral and of the time stepping
runs in the CUDA kernels behind the C ABI of include/best.h; this module only
marshals arguments.  PyTorch provides device memory and streams.  There is no
CPU fallback: if libbest.so is missing or no CUDA device is present, calls
fail.
"""
import ctypes

import numpy as np

from . import _lib
from ._lib import BestError, check

__all__ = ["Collision", "BestError", "build", "chunk_bounds", "config_from_problem", "fixed_sample_collision",
           "vegas_iteration_noalloc"]


def build(verbose=False, force=False):
    from .buildlib import build as _build
    return _build(verbose=verbose, force=force)


def chunk_bounds(cost, grid):
    """Chunk starts of the dynamic work partition of one VEGAS iteration of
    estimated cost `cost` over `grid` persistent CTAs (best_chunk_bounds;
    host arithmetic, no device needed): int64 array of chunks + 1 entries,
    0 first and cost last."""
    lib = _lib.load()
    k = ctypes.c_int32(0)
    lib.best_chunk_bounds(int(cost), int(grid), None, 0, ctypes.byref(k))     # asks for the count
    if k.value <= 0:
        raise BestError(f"best_chunk_bounds: {lib.best_last_error(None).decode()}")
    out = np.zeros(k.value + 1, dtype=np.int64)
    st = lib.best_chunk_bounds(int(cost), int(grid), out.ctypes.data_as(ctypes.c_void_p), len(out), ctypes.byref(k))
    if st != 0:
        raise BestError(f"best_chunk_bounds: {lib.best_last_error(None).decode()}")
    return out


def config_from_problem(problem, precision):
    """best_config for a ``workloads.Problem`` (plus the arrays it points to,
    which must outlive the init call)."""
    keep = []
    g = problem.grid
    sp = (_lib.best_species * len(problem.species))()
    for k, s in enumerate(problem.species):
        sp[k].stat = int(s.stat)
        sp[k].mass0 = float(s.mass0)
        sp[k].mass1 = float(s.mass1)
        tab = getattr(s, "mass_table", None)
        if tab is not None:
            if not 2 <= len(tab) <= _lib.MAX_MASS_KNOTS:
                raise BestError(f"species {s.name}: a mass table needs 2..{_lib.MAX_MASS_KNOTS} knots")
            sp[k].n_mass_knots = len(tab)
            for j, (tj, mj) in enumerate(tab):
                sp[k].mass_t[j] = float(tj)
                sp[k].mass_m[j] = float(mj)
    pr = (_lib.best_process * len(problem.processes))()
    for k, p in enumerate(problem.processes):
        legs = tuple(p.species_in) + tuple(p.species_out)
        if len(legs) > _lib.MAX_LEGS:
            raise BestError(f"process {p.name}: more than {_lib.MAX_LEGS} legs")
        pr[k].n_in = len(p.species_in)
        pr[k].n_out = len(p.species_out)
        for j, s in enumerate(legs):
            pr[k].species[j] = int(s)
        pr[k].coupling = float(p.coupling)
        pr[k].sigma_E = float(p.sigma_E)
        pr[k].neval = int(p.neval)
        if p.neval_per_point is not None:
            arr = (ctypes.c_int64 * len(p.neval_per_point))(*[int(v) for v in p.neval_per_point])
            keep.append(arr)
            pr[k].neval_per_point = ctypes.cast(arr, ctypes.POINTER(ctypes.c_int64))
        pr[k].nitn = int(p.nitn)
        pr[k].nbins = int(p.nbins)
        pr[k].alpha = float(p.alpha)
        pr[k].width_mode = int(getattr(p, "width_mode", 0))
        pr[k].width = float(getattr(p, "width", 0.01))
        pr[k].width_rel_lo = float(getattr(p, "width_rel_lo", 1e-3))
        pr[k].width_rel_hi = float(getattr(p, "width_rel_hi", 1e-2))
        pr[k].width_factor = float(getattr(p, "width_factor", 1.25))
        pr[k].width_min = float(getattr(p, "width_min", 1e-4))
        pr[k].width_max = float(getattr(p, "width_max", 0.2))
        pr[k].strat = int(getattr(p, "strat", 0))
        pr[k].strat_max_hcubes = int(getattr(p, "strat_max_hcubes", 64))
        pr[k].strat_beta = float(getattr(p, "strat_beta", 0.75))
        for j, c in enumerate(getattr(p, "me_coef", (1.0, 0.0, 0.0, 0.0))):
            pr[k].me_coef[j] = float(c)
        pr[k].budget = int(getattr(p, "budget", 0))
        pr[k].sides = int(getattr(p, "sides", 0))
        pr[k].neval_min = int(getattr(p, "neval_min", 0))
        pr[k].neval_max = int(getattr(p, "neval_max", 0))
    cfg = _lib.best_config()
    cfg.grid.n = int(g.n)
    cfg.grid.log_spaced = 1 if g.log_spaced else 0
    cfg.grid.q_min = float(g.q_min)
    cfg.grid.q_max = float(g.q_max)
    cfg.n_species = len(problem.species)
    cfg.n_processes = len(problem.processes)
    cfg.species = ctypes.cast(sp, ctypes.POINTER(_lib.best_species))
    cfg.processes = ctypes.cast(pr, ctypes.POINTER(_lib.best_process))
    cfg.precision = int(precision)
    cfg.tail_points = int(problem.tail_points)
    cfg.seed = int(problem.seed) & 0xFFFFFFFFFFFFFFFF
    cfg.e_cut = float(problem.e_cut)
    if problem.expansion is not None:
        cfg.expansion = 1
        cfg.a0 = float(problem.expansion.a0)
        cfg.t0 = float(problem.expansion.t0)
    else:
        cfg.expansion = 0
        cfg.a0 = 1.0
        cfg.t0 = 1.0
    cfg.eps_dt = float(problem.eps_dt)
    keep += [sp, pr]
    return cfg, keep


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p(0)


def _stream(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _require(t, n, name):
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
        raise BestError(f"{name} must be a contiguous CUDA float64 tensor")
    if t.numel() != n:
        raise BestError(f"{name} must have {n} elements, got {t.numel()}")


def _require_opt(t, n, name):
    """As _require, for an optional output (None: the library's own buffer)."""
    if t is not None:
        _require(t, n, name)


def _require_time(t_dev, dt_dev):
    """t and dt of a device-side step: one-element CUDA float64 tensors."""
    _require(t_dev, 1, "t")
    _require(dt_dev, 1, "dt")


class Collision:
    """One context of libbest: the tasks, VEGAS maps and device state of a
    problem.  ``precision``: workloads.PREC_FP64 or PREC_FP32."""

    def __init__(self, problem, precision, points=None):
        import torch
        if not torch.cuda.is_available():
            raise BestError("a CUDA device is required")
        torch.cuda.init()
        self.lib = _lib.load()
        self.problem = problem
        self.precision = precision
        self.n_species = len(problem.species)
        self.n_grid = problem.grid.n
        cfg, keep = config_from_problem(problem, precision)
        if points is not None:
            # a shard: the tasks of grid points [lo, hi) only (see dist.sharded_step)
            cfg.point_lo, cfg.point_hi = int(points[0]), int(points[1])
        self.points = (0, problem.grid.n) if points is None else (int(points[0]), int(points[1]))
        ctx = ctypes.c_void_p()
        check(self.lib.best_collision_init(ctypes.byref(cfg), ctypes.byref(ctx)))
        del keep
        self.ctx = ctx
        self.n_tasks = self.lib.best_num_tasks(ctx)
        self.n_side = self.lib.best_num_side_integrals(ctx)

    # -- the hot path ---------------------------------------------------------
    def eval(self, f, t=0.0, C=None, err=None, stream=None):
        """C[f] and its MC error at time t; f: (n_species, n_grid) float64 CUDA."""
        import torch
        n = self.n_species * self.n_grid
        _require(f, n, "f")
        _require_opt(C, n, "C")
        _require_opt(err, n, "err")
        if C is None:
            C = torch.empty_like(f)
        if err is None:
            err = torch.empty_like(f)
        check(self.lib.best_collision_eval(self.ctx, _ptr(f), float(t), _ptr(C), _ptr(err),
                                           _stream(stream)), self.ctx)
        return C, err

    def step_euler(self, logf, t_dev, dt_dev, C=None, stream=None):
        _require(logf, self.n_species * self.n_grid, "logf")
        _require_time(t_dev, dt_dev)
        _require_opt(C, self.n_species * self.n_grid, "C")
        check(self.lib.best_step_euler(self.ctx, _ptr(logf), _ptr(t_dev), _ptr(dt_dev), _ptr(C),
                                       _stream(stream)), self.ctx)

    def eval_log(self, logf, t=0.0, C=None, err=None, stream=None):
        """eval from log f (the sweep exponentiates on the device)."""
        import torch
        n = self.n_species * self.n_grid
        _require(logf, n, "logf")
        _require_opt(C, n, "C")
        _require_opt(err, n, "err")
        if C is None:
            C = torch.empty_like(logf)
        if err is None:
            err = torch.empty_like(logf)
        check(self.lib.best_collision_eval_log(self.ctx, _ptr(logf), float(t), _ptr(C), _ptr(err), _stream(stream)),
              self.ctx)
        return C, err

    def step_stage(self, method, stage, logf, k1, t_dev, dt_dev, k2=None, fstar=None, stream=None):
        """One stage of an Euler (method 0) or Heun (method 1) step from an
        assembled C (best_step_stage)."""
        n = self.n_species * self.n_grid
        _require(logf, n, "logf")
        _require(k1, n, "k1")
        _require_opt(k2, n, "k2")
        _require_opt(fstar, n, "fstar")
        _require_time(t_dev, dt_dev)
        check(self.lib.best_step_stage(self.ctx, int(method), int(stage), _ptr(logf), _ptr(k1), _ptr(k2), _ptr(fstar),
                                       _ptr(t_dev), _ptr(dt_dev), _stream(stream)), self.ctx)

    def step_heun(self, logf, t_dev, dt_dev, C=None, stream=None):
        _require(logf, self.n_species * self.n_grid, "logf")
        _require_time(t_dev, dt_dev)
        _require_opt(C, self.n_species * self.n_grid, "C")
        check(self.lib.best_step_heun(self.ctx, _ptr(logf), _ptr(t_dev), _ptr(dt_dev), _ptr(C),
                                      _stream(stream)), self.ctx)

    def evolve(self, logf, t_dev, dt_dev, n_steps, dt_request, method="heun", stream=None):
        """n_steps Euler/Heun steps replayed from a CUDA graph captured on
        `stream` (a created torch.cuda.Stream; defaults to a private one)."""
        import torch
        _require(logf, self.n_species * self.n_grid, "logf")
        _require_time(t_dev, dt_dev)
        if stream is None:
            if getattr(self, "_graph_stream", None) is None:
                self._graph_stream = torch.cuda.Stream()
            stream = self._graph_stream
            stream.wait_stream(torch.cuda.current_stream())
        m = {"euler": 0, "heun": 1}[method]
        check(self.lib.best_evolve(self.ctx, m, int(n_steps), _ptr(logf), _ptr(t_dev), _ptr(dt_dev),
                                   float(dt_request), ctypes.c_void_p(stream.cuda_stream)), self.ctx)
        torch.cuda.current_stream().wait_stream(stream)

    def autotune(self, f, t=0.0, stream=None):
        """Pick the fastest sample-kernel variant on this workload; returns
        the chosen CTAs per SM.  Maps, scales and counter are preserved."""
        _require(f, self.n_species * self.n_grid, "f")
        mb = ctypes.c_int32(0)
        check(self.lib.best_autotune(self.ctx, _ptr(f), float(t), ctypes.byref(mb), _stream(stream)), self.ctx)
        return mb.value

    def vjp(self, f, v, t=0.0, stream=None):
        """(C~, dL/df, dL/dm, dL/dcoupling) of L = sum(v * C~) for the
        fixed-sample integral C~ (one iteration on the current maps)."""
        import torch
        n = self.n_species * self.n_grid
        _require(f, n, "f")
        _require(v, n, "v")
        C = torch.empty_like(f)
        gf = torch.empty_like(f)
        gm = torch.empty(self.n_species, dtype=torch.float64, device=f.device)
        gl = torch.empty(len(self.problem.processes), dtype=torch.float64, device=f.device)
        check(self.lib.best_collision_vjp(self.ctx, _ptr(f), float(t), _ptr(v), _ptr(C), _ptr(gf), _ptr(gm),
                                          _ptr(gl), _stream(stream)), self.ctx)
        return C, gf, gm, gl

    def jvp(self, f, u, t=0.0, stream=None):
        """(C~, J u) for J = dC~/df of the fixed-sample integral (the same
        samples as vjp)."""
        import torch
        n = self.n_species * self.n_grid
        _require(f, n, "f")
        _require(u, n, "u")
        C = torch.empty_like(f)
        JU = torch.empty_like(f)
        check(self.lib.best_collision_jvp(self.ctx, _ptr(f), float(t), _ptr(u), _ptr(C), _ptr(JU), _stream(stream)),
              self.ctx)
        return C, JU

    def step_implicit_euler(self, logf, t, dt, train=True, tol=None, max_newton=8, krylov_dim=24,
                            krylov_rtol=1e-6, stream=None, raise_on_failure=True):
        """Backward Euler step of log f in place (Newton-Krylov on the
        fixed-sample integral at t + dt).  tol defaults to 1e-10 (FP64) or
        1e-6 (FP32) in ||R||_inf.  Returns a dict of the solver's counts;
        when Newton does not converge, logf is unchanged and BestError is
        raised (or, with raise_on_failure=False, the dict has converged=False)."""
        n = self.n_species * self.n_grid
        _require(logf, n, "logf")
        if tol is None:
            tol = 1e-6 if self.precision == 1 else 1e-10          # 1: FP32
        info = (ctypes.c_double * 5)()
        st = self.lib.best_step_implicit_euler(self.ctx, _ptr(logf), float(t), float(dt), int(bool(train)),
                                               float(tol), int(max_newton), int(krylov_dim), float(krylov_rtol),
                                               info, _stream(stream))
        out = {"newton": int(info[0]), "krylov": int(info[1]), "residual": info[2], "converged": info[3] == 1.0,
               "halvings": int(info[4])}
        if st != 0 and (raise_on_failure or out["converged"] or info[0] == 0):
            check(st, self.ctx)
        return out

    def moments(self, f, t=0.0, stream=None):
        """(n, rho): number and energy density of every species (device tensors)."""
        import torch
        _require(f, self.n_species * self.n_grid, "f")
        n = torch.empty(self.n_species, dtype=torch.float64, device=f.device)
        rho = torch.empty_like(n)
        check(self.lib.best_moments(self.ctx, _ptr(f), float(t), _ptr(n), _ptr(rho), _stream(stream)), self.ctx)
        return n, rho

    def strata(self, task):
        """(M, H, m): strata per dimension, hypercubes and items per
        hypercube of a stratified task (H = 0 and m = None otherwise)."""
        M = ctypes.c_int32(0)
        H = ctypes.c_int32(0)
        check(self.lib.best_get_strata(self.ctx, int(task), ctypes.byref(M), ctypes.byref(H), None), self.ctx)
        if H.value == 0:
            return M.value, 0, None
        m = np.zeros(H.value, dtype=np.int32)
        check(self.lib.best_get_strata(self.ctx, int(task), None, None, m.ctypes.data_as(ctypes.c_void_p)),
              self.ctx)
        return M.value, H.value, m

    def species_masses(self, t):
        """m_s(t) of every species as the library evaluates it (numpy)."""
        m = (ctypes.c_double * self.n_species)()
        check(self.lib.best_species_masses(self.ctx, float(t), m), self.ctx)
        return np.array(m[:])

    def widths(self):
        """(w, rel): the fractional Gaussian width of every process as the
        next evaluation uses it, and the relative error that last set it."""
        P = len(self.problem.processes)
        w = (ctypes.c_double * P)()
        r = (ctypes.c_double * P)()
        check(self.lib.best_get_widths(self.ctx, w, r), self.ctx)
        return np.array(w[:]), np.array(r[:])

    def set_widths(self, w):
        P = len(self.problem.processes)
        arr = (ctypes.c_double * P)(*[float(x) for x in w])
        check(self.lib.best_set_widths(self.ctx, arr), self.ctx)

    def save_state(self):
        """Maps, scales, counter and time state as bytes (see checkpoint.py)."""
        n = self.lib.best_state_size(self.ctx)
        buf = ctypes.create_string_buffer(n)
        check(self.lib.best_save_state(self.ctx, buf, n), self.ctx)
        return buf.raw

    def load_state(self, blob):
        buf = ctypes.create_string_buffer(bytes(blob), len(blob))
        check(self.lib.best_load_state(self.ctx, buf, len(blob)), self.ctx)

    # -- inspection -------------------------------------------------------------
    def check(self, stream=None):
        check(self.lib.best_check(self.ctx, _stream(stream)), self.ctx)

    def task_results(self, stream=None):
        mean = np.zeros(self.n_tasks)
        err = np.zeros(self.n_tasks)
        check(self.lib.best_get_task_results(self.ctx, mean.ctypes.data_as(ctypes.c_void_p),
                                             err.ctypes.data_as(ctypes.c_void_p), _stream(stream)), self.ctx)
        return mean, err

    def launch_shape(self):
        """(CTAs per SM, threads per CTA, samples per lane per step) of the sample kernel."""
        a, b, c = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        check(self.lib.best_launch_shape(self.ctx, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)), self.ctx)
        return a.value, b.value, c.value

    def budgets(self, stream=None):
        """Samples per iteration of every task in the next sweep (int64 array)."""
        out = np.zeros(self.n_tasks, dtype=np.int64)
        check(self.lib.best_get_budgets(self.ctx, out.ctypes.data_as(ctypes.c_void_p), _stream(stream)), self.ctx)
        return out

    def maps(self):
        stride = self.lib.best_map_stride(self.ctx)
        out = np.zeros(self.n_tasks * stride)
        check(self.lib.best_get_maps(self.ctx, out.ctypes.data_as(ctypes.c_void_p)), self.ctx)
        return out.reshape(self.n_tasks, stride)

    def set_maps(self, edges):
        edges = np.ascontiguousarray(edges, dtype=np.float64)
        check(self.lib.best_set_maps(self.ctx, edges.ctypes.data_as(ctypes.c_void_p)), self.ctx)

    @property
    def call_counter(self):
        c = ctypes.c_uint32()
        check(self.lib.best_get_call_counter(self.ctx, ctypes.byref(c)), self.ctx)
        return c.value

    @call_counter.setter
    def call_counter(self, value):
        check(self.lib.best_set_call_counter(self.ctx, int(value)), self.ctx)

    def profile(self, enable=True):
        check(self.lib.best_profile_enable(self.ctx, 1 if enable else 0), self.ctx)

    def profile_read(self):
        """(summed sample-kernel milliseconds, launches) since the last read."""
        ms = ctypes.c_double()
        n = ctypes.c_int64()
        check(self.lib.best_profile_read(self.ctx, ctypes.byref(ms), ctypes.byref(n)), self.ctx)
        return ms.value, n.value

    def partition_groups(self, iteration):
        """Sample groups of every task covered by the work partition of VEGAS
        iteration `iteration` (int64 array; -1 where a task's segments do not
        tile its groups exactly, 0 for inactive tasks)."""
        out = np.zeros(self.n_tasks, dtype=np.int64)
        check(self.lib.best_partition_groups(self.ctx, int(iteration), out.ctypes.data_as(ctypes.c_void_p)),
              self.ctx)
        return out

    def sweep_samples(self, iteration=-1):
        """Integrand evaluations per sweep (or in one VEGAS iteration)."""
        return self.lib.best_sweep_samples(self.ctx, int(iteration))

    def last_launch_count(self):
        return self.lib.best_last_launch_count(self.ctx)

    def close(self):
        if getattr(self, "ctx", None) is not None and self.ctx.value:
            self.lib.best_collision_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _autograd_function():
    import torch

    class FixedSampleCollision(torch.autograd.Function):
        """C~(f, m, lambda): the fixed-sample collision integral of a context
        (one VEGAS iteration per task on its current maps, common random
        numbers).  Forward and backward both run best_collision_vjp; the
        backward pass recomputes the samples instead of storing them."""

        @staticmethod
        def forward(ctx, col, f, masses, couplings, t):
            zero = torch.zeros_like(f)
            C, _, _, _ = col.vjp(f.detach().contiguous(), zero, t)
            ctx.col = col
            ctx.t = t
            ctx.save_for_backward(f)
            return C

        @staticmethod
        def backward(ctx, grad_C):
            (f,) = ctx.saved_tensors
            _, gf, gm, gl = ctx.col.vjp(f.detach().contiguous(), grad_C.contiguous(), ctx.t)
            return None, gf, gm, gl, None

    return FixedSampleCollision


_FSC = None


def fixed_sample_collision(col, f, t=0.0, masses=None, couplings=None):
    """Differentiable C~ of context `col` at grid values f (CUDA float64,
    (n_species, n_grid)).  `masses` (n_species,) and `couplings`
    (n_processes,) are optional tensors that must equal the context's m_s(t)
    and couplings; pass them with requires_grad to receive dL/dm, dL/dlambda."""
    import torch
    global _FSC
    if _FSC is None:
        _FSC = _autograd_function()
    prob = col.problem
    m_now = torch.tensor(col.species_masses(t), dtype=torch.float64, device=f.device)
    lam_now = torch.tensor([p.coupling for p in prob.processes], dtype=torch.float64, device=f.device)
    if masses is None:
        masses = m_now
    elif not torch.allclose(masses.detach(), m_now, rtol=1e-12, atol=0):
        raise BestError("masses must equal the context's m_s(t)")
    if couplings is None:
        couplings = lam_now
    elif not torch.allclose(couplings.detach(), lam_now, rtol=1e-12, atol=0):
        raise BestError("couplings must equal the context's couplings")
    return _FSC.apply(col, f, masses, couplings, float(t))


def _task_process(problem, task):
    """The process whose side integral holds task id `task` (tasks are
    numbered (side integral * n_grid + point) * 2 + term, side integrals by
    process, then side, then species)."""
    n = problem.grid.n
    si = task // (2 * n) if task >= 0 else -1
    k = 0
    for p in problem.processes:
        sym = sorted(p.species_in) == sorted(p.species_out)
        count = len(set(p.species_in)) + (0 if sym else len(set(p.species_out)))
        if 0 <= si < k + count:
            return p
        k += count
    raise BestError(f"task {task} out of range")


def vegas_iteration_noalloc(problem, precision, task, f, t, edges, out, iteration=0, call=0, stream=None):
    """One VEGAS iteration of one task through best_vegas_iteration_noalloc,
    which allocates no device memory (its scratch is a static device array).
    f: (n_species * n_grid) grid values; edges: the task's map,
    D * (nbins + 1) values; out: 2 + D * nbins values (sum w, sum w^2, the
    per-increment sums of w^2); all contiguous CUDA float64 tensors."""
    p = _task_process(problem, task)
    D = 3 * (len(p.species_in) + len(p.species_out) - 2)
    _require(f, len(problem.species) * problem.grid.n, "f")
    _require(edges, D * (p.nbins + 1), "edges")
    _require(out, 2 + D * p.nbins, "out")
    lib = _lib.load()
    cfg, keep = config_from_problem(problem, precision)
    st = lib.best_vegas_iteration_noalloc(ctypes.byref(cfg), int(task), _ptr(f), float(t), _ptr(edges),
                                          int(iteration) & 0xFFFFFFFF, int(call) & 0xFFFFFFFF, _ptr(out),
                                          _stream(stream))
    del keep
    if st != 0:
        raise BestError(f"best_vegas_iteration_noalloc: {lib.best_last_error(None).decode()}")
    return out
