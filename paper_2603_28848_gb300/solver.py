"""A solver object with the paper's way of setting up a run (App. D): a
momentum grid, species registered with an initial distribution, statistics
and mass, processes registered by their initial and final species, then
repeated time steps; checkpoints hold everything needed to resume.

It only assembles a ``workloads.Problem`` and sequences libbest calls
(``Collision``); every step of the computation runs in the library.

    s = Solver(q_min=0.05, q_max=25.0, n_grid=96)
    s.initialize_species("chi", lambda q: 0.4 * np.exp(-(q - 2.0) ** 2), stat="boson", mass=0.7)
    s.add_process("chichi", ["chi", "chi"], ["chi", "chi"], lambda k, g: g * g * np.ones(k.shape[-1]),
                  coupling=0.5, neval=4 * 10**5, delta_width=0.02)
    while s.current_time < 40.0:
        s.evolve_step(dt=0.5, method="heun")

Differences from the paper's interface, by necessity of running on the GPU:
the matrix element is |M|^2 = coupling^2 P(s) with P a cubic in the initial
state's invariant mass squared (a callable in the paper's form is accepted
and reduced to P by probing it, ``matrix_element_polynomial``); a mass
may depend on time linearly (``set_mass_linear``) or piecewise linearly
through up to eight knots (``set_mass_table``); ``set_mass_func`` samples a
callable at given times into such a table.
"""
import numpy as np

import workloads as W

_STATS = {"boson": W.STAT_BE, "be": W.STAT_BE, "fermion": W.STAT_FD, "fd": W.STAT_FD,
          "maxwell": W.STAT_MB, "mb": W.STAT_MB, "classical": W.STAT_MB}


def matrix_element_polynomial(fn, coupling, m_in, m_out, p_max, n_probe=256, seed=20260328):
    """Coefficients (c0, c1, c2, c3) with fn = coupling^2 (c0 + c1 s + c2 s^2
    + c3 s^3) for a matrix element given as the paper's callable
    fn(momenta, coupling) -> |M|^2 per sample (Sec. 3A).

    Reading of the callable's argument: momenta has shape (n_legs, 4, N),
    row k = (E, px, py, pz) of leg k, the initial legs first, N samples
    (the paper's example reads N from momenta.shape[2]).  The callable is
    probed on N random configurations (momenta up to p_max, directions
    uniform, on-shell energies; the final legs drawn independently); s is
    the initial state's invariant mass squared.  A callable that is not a
    polynomial of degree <= 3 in s alone (it depends on final momenta or
    angles, or grows faster) cannot run in the kernels and raises
    ValueError."""
    if not coupling:
        raise ValueError("the coupling must be non-zero to separate |M|^2 = coupling^2 P(s)")
    rng = np.random.default_rng(seed)
    legs = []
    for m in list(m_in) + list(m_out):
        p = rng.uniform(0.0, p_max, n_probe)
        ct = rng.uniform(-1.0, 1.0, n_probe)
        ph = rng.uniform(0.0, 2.0 * np.pi, n_probe)
        st = np.sqrt(1.0 - ct * ct)
        legs.append(np.stack([np.sqrt(p * p + m * m), p * st * np.cos(ph), p * st * np.sin(ph), p * ct]))
    momenta = np.stack(legs)
    vals = np.broadcast_to(np.asarray(fn(momenta, coupling), dtype=np.float64), (n_probe,)) / coupling ** 2
    if not np.all(np.isfinite(vals)):
        raise ValueError("the matrix element is not finite on the probe configurations")
    tot = momenta[:len(m_in)].sum(axis=0)
    s = tot[0] ** 2 - tot[1] ** 2 - tot[2] ** 2 - tot[3] ** 2
    scale = max(float(np.max(np.abs(s))), 1e-300)
    a = np.polynomial.polynomial.polyfit(s / scale, vals, 3)
    resid = float(np.max(np.abs(np.polynomial.polynomial.polyval(s / scale, a) - vals)))
    if resid > 1e-8 * max(float(np.max(np.abs(vals))), 1e-300):
        raise ValueError("the matrix element is not a cubic polynomial of the initial state's s alone "
                         f"(fit residual {resid:.3g}); give P(s) coefficients instead")
    c = a / scale ** np.arange(4)
    c[np.abs(a) <= 1e-12 * max(float(np.max(np.abs(a))), 1e-300)] = 0.0
    return tuple(float(x) for x in c)


class Solver:
    def __init__(self, q_min, q_max, n_grid, log_spaced=True, precision="fp32", seed=0, eps_dt=0.3,
                 tail_points=4, e_cut=1e-12):
        self.grid = W.Grid(int(n_grid), float(q_min), float(q_max), bool(log_spaced))
        self.precision = W.PREC_FP32 if precision in ("fp32", W.PREC_FP32) else W.PREC_FP64
        self.seed = int(seed)
        self.eps_dt = float(eps_dt)
        self.tail_points = int(tail_points)
        self.e_cut = float(e_cut)
        self.current_time = 1.0
        self.expansion = None
        self._species = []          # (name, Species, initial grid values)
        self._processes = []
        self._col = None
        self._logf = self._t = self._dt = None
        self.history = None          # what load_checkpoint found saved beside the state

    # -- set-up ---------------------------------------------------------------
    def q(self):
        """The comoving momentum grid (numpy)."""
        return W.grid_points(self.grid)

    def initialize_species(self, name, init_f, stat="boson", mass=0.0, mass_slope=0.0):
        """Register a species with f(q) on the grid from ``init_f`` (a callable
        of the comoving momenta or an array), statistics boson / fermion /
        maxwell and mass m(t) = mass + mass_slope t."""
        if any(n == name for n, _, _ in self._species):
            raise ValueError(f"species {name!r} is already registered")
        key = str(stat).lower()
        if key not in _STATS:
            raise ValueError(f"unknown statistics {stat!r} (boson, fermion or maxwell)")
        q = W.grid_points(self.grid)
        f = np.asarray(init_f(q) if callable(init_f) else init_f, dtype=np.float64).reshape(-1)
        if f.shape != q.shape or not np.all(np.isfinite(f)) or np.any(f <= 0.0):
            raise ValueError(f"initial distribution of {name!r} must be finite and positive on the {len(q)} points")
        self._species.append((name, W.Species(name, _STATS[key], float(mass), float(mass_slope)), f))
        self._invalidate()

    def set_mass_linear(self, name, mass, slope=0.0):
        """m(t) = mass + slope t for a registered species."""
        k = self._index(name)
        n, sp, f = self._species[k]
        self._species[k] = (n, W.Species(n, sp.stat, float(mass), float(slope)), f)
        self._invalidate()

    def set_mass_table(self, name, times, masses):
        """m(t) of a registered species as the straight lines through the knots
        (times[k], masses[k]) (2..8 knots, times increasing), constant
        beyond either end."""
        t = [float(x) for x in times]
        m = [float(x) for x in masses]
        if not 2 <= len(t) <= W.MAX_MASS_KNOTS or len(m) != len(t):
            raise ValueError(f"a mass table needs 2..{W.MAX_MASS_KNOTS} knots and one mass per time")
        if any(b <= a for a, b in zip(t[:-1], t[1:])) or any(not np.isfinite(x) or x < 0 for x in m):
            raise ValueError("mass knots need increasing times and finite masses >= 0")
        k = self._index(name)
        n, sp, f = self._species[k]
        self._species[k] = (n, W.Species(n, sp.stat, m[0], 0.0, tuple(zip(t, m))), f)
        self._invalidate()

    def set_mass_func(self, name, fn, times):
        """m(t) = fn(t) sampled at ``times`` (2..8 of them) and joined by
        straight lines."""
        self.set_mass_table(name, times, [float(fn(float(x))) for x in times])

    def add_process(self, name, initial, final, matrix_element=None, coupling=1.0, neval=10 ** 6,
                    delta_width=0.01, nitn=2, alpha=0.5, nbins=50, me_coef=None, **options):
        """Register initial -> final (species names).  ``matrix_element`` is
        the paper's callable |M|^2(momenta, coupling) (see
        ``matrix_element_polynomial``: it must be a cubic in the initial
        state's s), or the coefficients (c0, c1, c2, c3) of P(s) with
        |M|^2 = coupling^2 P(s), or None for |M|^2 = coupling^2 (also
        ``me_coef=``).  ``delta_width`` is the absolute width sigma_E of
        Eq. (11); ``options`` are further ``workloads.Process`` fields
        (width_mode, width, strat, ...)."""
        if matrix_element is not None and me_coef is not None:
            raise ValueError("give the matrix element either as matrix_element or as me_coef")
        sp_in = tuple(self._index(s) for s in initial)
        sp_out = tuple(self._index(s) for s in final)
        if callable(matrix_element):
            mass = [self._species[k][1].mass0 for k in sp_in + sp_out]
            me_coef = matrix_element_polynomial(matrix_element, float(coupling), mass[:len(sp_in)],
                                                mass[len(sp_in):], self.grid.q_max)
        elif matrix_element is not None:
            me_coef = matrix_element
        if me_coef is None:
            me_coef = (1.0, 0.0, 0.0, 0.0)
        me_coef = tuple(float(c) for c in me_coef) + (0.0,) * (4 - len(me_coef))
        if len(me_coef) != 4:
            raise ValueError("P(s) has at most four coefficients (a cubic in s)")
        p = W.Process(name, sp_in, sp_out, float(coupling), float(delta_width), int(neval), int(nitn),
                      float(alpha), int(nbins), me_coef=me_coef, **options)
        self._processes.append(p)
        self._invalidate()

    def set_radiation_dominated(self, a0=1.0, t0=None):
        """a(t) = a0 (t / t0)^(1/2); t0 defaults to the current time."""
        self.expansion = W.Expansion(float(a0), float(self.current_time if t0 is None else t0))
        self._invalidate()

    def problem(self):
        if not self._species or not self._processes:
            raise ValueError("register at least one species and one process")
        return W.Problem(self.grid, tuple(s for _, s, _ in self._species), tuple(self._processes),
                         seed=self.seed, e_cut=self.e_cut, tail_points=self.tail_points,
                         expansion=self.expansion, eps_dt=self.eps_dt)

    # -- evolution ------------------------------------------------------------
    def evolve_step(self, dt, method="heun"):
        """One Euler or Heun step (Eq. (14)-(16)); returns the step used."""
        col = self._context()
        self._dt.fill_(float(dt))
        (col.step_heun if method == "heun" else col.step_euler)(self._logf, self._t, self._dt)
        self.current_time = float(self._t.item())
        return float(self._dt.item())

    def evolve(self, n_steps, dt, method="heun"):
        """n_steps steps replayed from a captured CUDA graph."""
        col = self._context()
        col.evolve(self._logf, self._t, self._dt, int(n_steps), float(dt), method)
        self.current_time = float(self._t.item())

    def distribution(self, name):
        """f of a species on the grid (numpy)."""
        k = self._index(name)
        if self._logf is None:
            return self._species[k][2].copy()
        return np.exp(self._logf[k].cpu().numpy())

    def densities(self):
        """{name: (n, rho)}: number and energy densities at the current time."""
        import torch
        col = self._context()
        n, rho = col.moments(torch.exp(self._logf).contiguous(), self.current_time)
        n, rho = n.cpu().numpy(), rho.cpu().numpy()
        return {name: (float(n[k]), float(rho[k])) for k, (name, _, _) in enumerate(self._species)}

    # -- checkpoints ------------------------------------------------------------
    def save_checkpoint(self, path, history=None):
        """Grid, species, processes, distributions, time and the library state
        (VEGAS maps, allocations, widths, counter) in one .npz file, plus an
        optional user history (anything JSON can hold; numpy arrays are
        stored as lists), returned as ``.history`` by ``load_checkpoint``."""
        import json
        col = self._context()
        spec = {"grid": vars(self.grid), "precision": self.precision, "seed": self.seed, "eps_dt": self.eps_dt,
                "tail_points": self.tail_points, "e_cut": self.e_cut,
                "expansion": None if self.expansion is None else vars(self.expansion),
                "species": [vars(s) for _, s, _ in self._species],
                "processes": [vars(p) for p in self._processes],
                "history": history}
        as_json = lambda o: o.tolist() if hasattr(o, "tolist") else float(o)
        np.savez(path, spec=np.frombuffer(json.dumps(spec, default=as_json).encode(), dtype=np.uint8),
                 logf=self._logf.cpu().numpy(), t=np.array([self.current_time]),
                 state=np.frombuffer(col.save_state(), dtype=np.uint8))

    @classmethod
    def load_checkpoint(cls, path):
        """A solver resumed from ``save_checkpoint``: its next steps continue
        the saved run bit for bit."""
        import json
        z = np.load(path)
        spec = json.loads(z["spec"].tobytes().decode())
        g = spec["grid"]
        s = cls(g["q_min"], g["q_max"], g["n"], g["log_spaced"], spec["precision"], spec["seed"], spec["eps_dt"],
                spec["tail_points"], spec["e_cut"])
        logf = z["logf"]
        for k, sp in enumerate(spec["species"]):
            s._species.append((sp["name"], W.Species(**sp), np.exp(logf[k])))
        for p in spec["processes"]:
            p = dict(p)
            for key in ("species_in", "species_out", "me_coef"):
                p[key] = tuple(p[key])
            if p.get("neval_per_point") is not None:
                p["neval_per_point"] = tuple(p["neval_per_point"])
            s._processes.append(W.Process(**p))
        if spec["expansion"] is not None:
            s.expansion = W.Expansion(**spec["expansion"])
        s.current_time = float(z["t"][0])
        s.history = spec.get("history")
        col = s._context()
        col.load_state(z["state"].tobytes())
        s._logf.copy_(s._to_dev(logf))
        return s

    def close(self):
        if self._col is not None:
            self._col.close()
            self._col = None

    # -- internals --------------------------------------------------------------
    def _index(self, name):
        for k, (n, _, _) in enumerate(self._species):
            if n == name:
                return k
        raise ValueError(f"unknown species {name!r}")

    def _invalidate(self):
        if self._col is not None:
            # keep the evolved distributions, rebuild the context (maps start afresh)
            for k, (n, sp, _) in enumerate(self._species):
                if self._logf is not None and k < self._logf.shape[0]:
                    self._species[k] = (n, sp, np.exp(self._logf[k].cpu().numpy()))
            self._col.close()
            self._col = None
            self._logf = None

    def _to_dev(self, a):
        import torch
        return torch.tensor(np.asarray(a, dtype=np.float64), device="cuda").contiguous()

    def _context(self):
        if self._col is None:
            import torch
            from . import Collision
            self._col = Collision(self.problem(), self.precision)
            self._logf = self._to_dev(np.log(np.stack([f for _, _, f in self._species])))
            self._t = torch.tensor([self.current_time], dtype=torch.float64, device="cuda")
            self._dt = torch.tensor([0.0], dtype=torch.float64, device="cuda")
        return self._col
