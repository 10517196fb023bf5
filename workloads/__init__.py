"""Seeded synthetic inputs for the collision-integral hot path.

This module holds plain problem descriptions (momentum grid, species,
processes, sample budgets, seeds) and the initial distributions f0(q) of the
five benchmark workloads.  It holds none of the method's arithmetic: no
kinematics, sampling, integration, interpolation or time stepping.  Both the
CPU oracle (``oracle/``) and the CUDA library binding consume these objects,
and neither imports the other.

Problem layout (Sec. 3A of the paper):
  * one comoving momentum grid shared by all species, log or linear spaced
    over [q_min, q_max] with n points;
  * species with a statistics label (MB, BE, FD) and a mass
    m(t) = mass0 + mass1 * t or a piecewise-linear table of (t, m) knots
    (the time-dependent mass of Sec. 3A);
  * processes n_in -> n_out given by species index lists, a constant
    |M|^2 = coupling^2, the Gaussian width sigma_E of Eq. (11) and the VEGAS
    parameters neval (samples per iteration per task), nitn, alpha, nbins;
  * optional radiation-dominated expansion a(t) = a0 (t/t0)^(1/2) (Sec. 3E).
"""
from __future__ import annotations

from dataclasses import dataclass, field, replace
from typing import Optional, Tuple

import numpy as np

STAT_MB = 0
STAT_BE = 1
STAT_FD = 2
STAT_NAMES = {STAT_MB: "MB", STAT_BE: "BE", STAT_FD: "FD"}

PREC_FP64 = 0
PREC_FP32 = 1

WIDTH_ABSOLUTE = 0
WIDTH_FRACTIONAL = 1
WIDTH_ADAPTIVE = 2


@dataclass(frozen=True)
class Grid:
    n: int
    q_min: float
    q_max: float
    log_spaced: bool = True


MAX_MASS_KNOTS = 8


@dataclass(frozen=True)
class Species:
    name: str
    stat: int
    mass0: float
    mass1: float = 0.0          # m(t) = mass0 + mass1 * t
    # Optional knots ((t_0, m_0), ..., (t_k, m_k)), t increasing, 2..8 of
    # them: m(t) is then the piecewise-linear interpolant, held constant
    # outside [t_0, t_k] (mass0 and mass1 are ignored).
    mass_table: Optional[Tuple[Tuple[float, float], ...]] = None

    def __post_init__(self):
        if self.mass_table is not None:
            tab = tuple((float(a), float(b)) for a, b in self.mass_table)
            object.__setattr__(self, "mass_table", tab)


@dataclass(frozen=True)
class Process:
    name: str
    species_in: Tuple[int, ...]
    species_out: Tuple[int, ...]
    coupling: float = 1.0       # constant |M|^2 = coupling^2
    sigma_E: float = 0.01
    neval: int = 10_000         # samples per iteration per task
    nitn: int = 2
    alpha: float = 0.5
    nbins: int = 50
    # Optional per-grid-point budgets (uneven budgets); overrides neval.
    neval_per_point: Optional[Tuple[int, ...]] = None
    # Width of the Gaussian of Eq. (11): WIDTH_ABSOLUTE uses sigma_E;
    # WIDTH_FRACTIONAL uses sigma = w (E_in + E_out) / 2 per sample with w =
    # width; WIDTH_ADAPTIVE also adapts w after every evaluation (App. C):
    # w / width_factor when the process's relative MC error is below
    # width_rel_lo, w * width_factor when above width_rel_hi, within
    # [width_min, width_max].
    width_mode: int = 0
    width: float = 0.01
    width_rel_lo: float = 1e-3
    width_rel_hi: float = 1e-2
    width_factor: float = 1.25
    width_min: float = 1e-4
    width_max: float = 0.2
    # Adaptive stratified sampling (VEGAS+): strat = 1 splits the map's unit
    # cube into at most strat_max_hcubes hypercubes whose sample counts adapt
    # as sigma_h^strat_beta; tasks then draw 8 floor(N / 8) samples.
    strat: int = 0
    strat_beta: float = 0.75
    strat_max_hcubes: int = 64
    # |M|^2 = coupling^2 * (c0 + c1 s + c2 s^2 + c3 s^3), s the squared
    # invariant mass of the initial state (constant |M|^2 by default).
    me_coef: Tuple[float, float, float, float] = (1.0, 0.0, 0.0, 0.0)
    # Variance-driven budgets: budget = 1 re-sets the per-task samples per
    # iteration after every sweep in proportion to the last sweep's relative
    # variance per sample, within [neval_min, neval_max], keeping the sum of
    # the configured budgets of the process (neval or neval_per_point).
    budget: int = 0
    neval_min: int = 0
    neval_max: int = 0
    # Side integrals evaluated (Eq. (7)): 0 all of them; 1 only those with
    # the observed leg initial; 2 only those with it final (e.g. C_3 alone of
    # a 2 -> 3 process, the paper's negative case of Sec. 5D).
    sides: int = 0


@dataclass(frozen=True)
class Expansion:
    """Radiation domination, a(t) = a0 * (t / t0)^(1/2)."""
    a0: float = 1.0
    t0: float = 1.0


@dataclass(frozen=True)
class Problem:
    grid: Grid
    species: Tuple[Species, ...]
    processes: Tuple[Process, ...]
    seed: int = 0
    e_cut: float = 1e-12        # samples with any E_k < e_cut are discarded
    tail_points: int = 4        # grid points used by each end fit of Eq. (13)
    expansion: Optional[Expansion] = None
    eps_dt: float = 0.3         # bound on max |dt C/f| of Eq. (16)

    def with_budget(self, neval=None, nitn=None):
        """Copy with every process's budget replaced (used for small cases)."""
        procs = []
        for p in self.processes:
            kw = {}
            if neval is not None:
                kw["neval"] = int(neval)
                kw["neval_per_point"] = None
            if nitn is not None:
                kw["nitn"] = int(nitn)
            procs.append(replace(p, **kw))
        return replace(self, processes=tuple(procs))


def grid_points(grid: Grid) -> np.ndarray:
    """Grid abscissae used only to tabulate the initial conditions below."""
    if grid.log_spaced:
        return np.geomspace(grid.q_min, grid.q_max, grid.n)
    return np.linspace(grid.q_min, grid.q_max, grid.n)


# ----------------------------------------------------------------------------
# The five workloads.  Readings of unstated items are listed beside each.
# ----------------------------------------------------------------------------

SEEDS = (0x5EED0001, 0x5EED0002, 0x5EED0003, 0x5EED0004, 0x5EED0005)


def c1_maxwell_2to2(n=32, neval=10_000, nitn=5):
    """2->2, one scalar, m=1, MB, |M|^2=1, 32 log points on [0.01,20],
    sigma_E=0.01, 50 bins, 5 iterations x 1e4 samples per point, FP64."""
    grid = Grid(n, 0.01, 20.0, True)
    sp = (Species("phi", STAT_MB, 1.0),)
    pr = (Process("phiphi->phiphi", (0, 0), (0, 0), 1.0, 0.01, neval, nitn, 0.5, 50),)
    prob = Problem(grid, sp, pr, seed=SEEDS[0])
    q = grid_points(grid)
    f0 = (0.5 * np.exp(-np.sqrt(q * q + 1.0) / 1.5))[None, :]
    return prob, f0


def c2_bose_2to2(n=128, neval=1_000_000, nitn=8):
    """2->2 massless and m=0.5 BE scalars, 128 log points on [1e-3,30],
    sigma_E=0.005, 1e6 samples x 8 iterations.  Reading: the two masses are
    two uncoupled species evaluated in one sweep (one phi phi -> phi phi
    process each).  f0 = BE(T=1) + 0.3 exp(-(p-3)^2 / (2*0.5^2))."""
    grid = Grid(n, 1e-3, 30.0, True)
    sp = (Species("phi0", STAT_BE, 0.0), Species("phi05", STAT_BE, 0.5))
    pr = (Process("phi0phi0->phi0phi0", (0, 0), (0, 0), 1.0, 0.005, neval, nitn, 0.5, 50),
          Process("phi05phi05->phi05phi05", (1, 1), (1, 1), 1.0, 0.005, neval, nitn, 0.5, 50))
    prob = Problem(grid, sp, pr, seed=SEEDS[1])
    q = grid_points(grid)
    bump = 0.3 * np.exp(-((q - 3.0) ** 2) / (2 * 0.5 ** 2))
    f0 = np.stack([1.0 / np.expm1(np.sqrt(q * q + m * m)) + bump for m in (0.0, 0.5)])
    return prob, f0


def c3_cannibal_2to3(n=256, neval=4_000_000, nitn=10, with_2to2=False):
    """2<->3 number-changing massive scalar, m=1, BE, 256 log points on
    [0.01,25], f0 = 0.2 exp(-E/0.7), sigma_E=0.01, 4e6 x 10.  Both pinned
    sides (C = 2 C2 + 3 C3).  with_2to2 adds the 6-dim phi phi -> phi phi."""
    grid = Grid(n, 0.01, 25.0, True)
    sp = (Species("phi", STAT_BE, 1.0),)
    pr = [Process("phiphi->phiphiphi", (0, 0), (0, 0, 0), 1.0, 0.01, neval, nitn, 0.5, 50)]
    if with_2to2:
        pr.append(Process("phiphi->phiphi", (0, 0), (0, 0), 1.0, 0.01, neval, nitn, 0.5, 50))
    prob = Problem(grid, sp, tuple(pr), seed=SEEDS[2])
    q = grid_points(grid)
    f0 = (0.2 * np.exp(-np.sqrt(q * q + 1.0) / 0.7))[None, :]
    return prob, f0


def c4_multi_species(n=512, nmin=100_000, nmax=10_000_000, nitn=2, variance_budgets=False):
    """Two coupled species (A: BE, m(t)=1+0.1t; B: FD, m=0.3) with
    AB->AB, AA->AAA and AAA->BB, radiation-dominated expansion
    (a0=1, t0=1), 512 log points on [0.01,25], uneven budgets
    N_i = nmin (nmax/nmin)^(i/(n-1)) per grid point; with variance_budgets
    that schedule is the first sweep's, and later sweeps re-set every task's
    budget from the last sweep's variance within [nmin, nmax], keeping the
    schedule's total."""
    grid = Grid(n, 0.01, 25.0, True)
    sp = (Species("A", STAT_BE, 1.0, 0.1), Species("B", STAT_FD, 0.3, 0.0))
    i = np.arange(n)
    sched = tuple(int(round(nmin * (nmax / nmin) ** (k / max(n - 1, 1)))) for k in i)
    vb = dict(budget=1, neval_min=nmin, neval_max=nmax) if variance_budgets else {}
    pr = (Process("AB->AB", (0, 1), (0, 1), 1.0, 0.01, nmin, nitn, 0.5, 50, sched, **vb),
          Process("AA->AAA", (0, 0), (0, 0, 0), 1.0, 0.01, nmin, nitn, 0.5, 50, sched, **vb),
          Process("AAA->BB", (0, 0, 0), (1, 1), 1.0, 0.01, nmin, nitn, 0.5, 50, sched, **vb))
    prob = Problem(grid, sp, pr, seed=SEEDS[3], expansion=Expansion(1.0, 1.0))
    q = grid_points(grid)
    fA = 1.0 / np.expm1(np.sqrt(q * q + 1.0))
    fB = 1.0 / (np.exp(np.sqrt(q * q + 0.09)) + 1.0)
    return prob, np.stack([fA, fB])


def c5_2to4(n=256, neval=2_000_000, nitn=2):
    """2->4 massive scalar (12-dim), m=1, BE, 256 log points on [0.01,25],
    f0 = 0.2 exp(-E/0.7), 2e6 samples per point."""
    grid = Grid(n, 0.01, 25.0, True)
    sp = (Species("phi", STAT_BE, 1.0),)
    pr = (Process("phiphi->4phi", (0, 0), (0, 0, 0, 0), 1.0, 0.01, neval, nitn, 0.5, 50),)
    prob = Problem(grid, sp, pr, seed=SEEDS[4])
    q = grid_points(grid)
    f0 = (0.2 * np.exp(-np.sqrt(q * q + 1.0) / 0.7))[None, :]
    return prob, f0


WORKLOADS = {
    "c1_maxwell_2to2": c1_maxwell_2to2,
    "c2_bose_2to2": c2_bose_2to2,
    "c3_cannibal_2to3": c3_cannibal_2to3,
    "c4_multi_species": c4_multi_species,
    "c5_2to4": c5_2to4,
}
