"""A solver object with the paper's way of setting up a run (App. D): a
momentum grid, species registered with an initial distribution, statistics
and mass, processes registered by their initial and final species, then
repeated time steps; checkpoints hold everything needed to resume.

It only assembles a ``workloads.Problem`` and sequences libbest calls
(``Collision``); every step of the computation runs in the library.

    s = Solver(q_min=0.1, q_max=20.0, n_grid=64)
    s.initialize_species("phi", lambda q: 1 / (1 + np.exp((q - 3) / 2)), stat="boson", mass=1.0)
    s.add_process("elastic", ["phi", "phi"], ["phi", "phi"], coupling=1.0, neval=10**6, delta_width=0.01)
    for _ in range(100):
        s.evolve_step(dt=1.0, method="heun")

Differences from the paper's interface, by necessity of running on the GPU:
the matrix element is |M|^2 = coupling^2 P(s) with P a cubic in the initial
state's invariant mass squared (``me_coef``), not a Python callable; a mass
may depend on time linearly (``set_mass_linear``) or piecewise linearly
through up to eight knots (``set_mass_table``); ``set_mass_func`` samples a
callable at given times into such a table.
"""
import numpy as np

import workloads as W

_STATS = {"boson": W.STAT_BE, "be": W.STAT_BE, "fermion": W.STAT_FD, "fd": W.STAT_FD,
          "maxwell": W.STAT_MB, "mb": W.STAT_MB, "classical": W.STAT_MB}


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

    def add_process(self, name, initial, final, coupling=1.0, neval=10 ** 6, delta_width=0.01, nitn=2,
                    alpha=0.5, nbins=50, me_coef=(1.0, 0.0, 0.0, 0.0), **options):
        """Register initial -> final (species names).  ``delta_width`` is the
        absolute width sigma_E of Eq. (11); ``options`` are further
        ``workloads.Process`` fields (width_mode, width, strat, ...)."""
        p = W.Process(name, tuple(self._index(s) for s in initial), tuple(self._index(s) for s in final),
                      float(coupling), float(delta_width), int(neval), int(nitn), float(alpha), int(nbins),
                      me_coef=tuple(float(c) for c in me_coef), **options)
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
    def save_checkpoint(self, path):
        """Grid, species, processes, distributions, time and the library state
        (VEGAS maps, allocations, widths, counter) in one .npz file."""
        import json
        col = self._context()
        spec = {"grid": vars(self.grid), "precision": self.precision, "seed": self.seed, "eps_dt": self.eps_dt,
                "tail_points": self.tail_points, "e_cut": self.e_cut,
                "expansion": None if self.expansion is None else vars(self.expansion),
                "species": [vars(s) for _, s, _ in self._species],
                "processes": [vars(p) for p in self._processes]}
        np.savez(path, spec=np.frombuffer(json.dumps(spec).encode(), dtype=np.uint8),
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
