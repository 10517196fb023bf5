"""The Solver's set-up (no GPU): species and processes become the same
workloads.Problem a direct construction gives, with clear errors for
unknown names, duplicates and bad initial data."""
import numpy as np
import pytest

import workloads as W
from paper_2603_28848_gb300.solver import Solver


def test_setup_builds_the_problem():
    s = Solver(q_min=0.01, q_max=25.0, n_grid=16, seed=7)
    s.initialize_species("A", lambda q: 1.0 / np.expm1(np.sqrt(q * q + 1.0)), stat="boson", mass=1.0,
                         mass_slope=0.1)
    s.initialize_species("B", lambda q: 1.0 / (np.exp(np.sqrt(q * q + 0.09)) + 1.0), stat="fermion", mass=0.3)
    s.add_process("AB->AB", ["A", "B"], ["A", "B"], coupling=1.0, neval=1000, delta_width=0.01)
    s.add_process("AA->AAA", ["A", "A"], ["A", "A", "A"], neval=2000, me_coef=(0.0, 1.0, 0.0, 0.0))
    s.set_radiation_dominated(a0=1.0)
    p = s.problem()
    assert p.grid == W.Grid(16, 0.01, 25.0, True)
    assert p.species == (W.Species("A", W.STAT_BE, 1.0, 0.1), W.Species("B", W.STAT_FD, 0.3, 0.0))
    assert p.processes[0].species_in == (0, 1) and p.processes[1].species_out == (0, 0, 0)
    assert p.processes[1].me_coef == (0.0, 1.0, 0.0, 0.0) and p.processes[1].neval == 2000
    assert p.expansion == W.Expansion(1.0, 1.0) and p.seed == 7
    assert np.allclose(s.distribution("B"), 1.0 / (np.exp(np.sqrt(s.q() ** 2 + 0.09)) + 1.0))


def test_setup_errors():
    s = Solver(0.1, 20.0, 8)
    s.initialize_species("phi", lambda q: np.exp(-q), stat="maxwell")
    with pytest.raises(ValueError):
        s.initialize_species("phi", lambda q: np.exp(-q))
    with pytest.raises(ValueError):
        s.initialize_species("chi", lambda q: -np.exp(-q))
    with pytest.raises(ValueError):
        s.initialize_species("chi", lambda q: np.exp(-q), stat="anyon")
    with pytest.raises(ValueError):
        s.add_process("bad", ["phi", "psi"], ["phi", "phi"])
    with pytest.raises(ValueError):
        Solver(0.1, 20.0, 8).problem()


def test_mass_table_and_func():
    s = Solver(0.1, 20.0, 8)
    s.initialize_species("phi", lambda q: np.exp(-q), stat="maxwell", mass=1.0)
    s.add_process("pp", ["phi", "phi"], ["phi", "phi"], neval=100)
    s.set_mass_table("phi", [1.0, 2.0, 4.0], [1.0, 0.2, 0.2])
    sp = s.problem().species[0]
    assert sp.mass_table == ((1.0, 1.0), (2.0, 0.2), (4.0, 0.2))
    s.set_mass_func("phi", lambda t: 2.0 / t, [1.0, 2.0, 4.0, 8.0])
    assert s.problem().species[0].mass_table == ((1.0, 2.0), (2.0, 1.0), (4.0, 0.5), (8.0, 0.25))
    s.set_mass_linear("phi", 0.5, 0.1)
    assert s.problem().species[0] == W.Species("phi", W.STAT_MB, 0.5, 0.1)
    for times, masses in (([1.0], [1.0]), ([1.0, 1.0], [1.0, 2.0]), ([2.0, 1.0], [1.0, 1.0]),
                          ([1.0, 2.0], [1.0, -1.0]), (list(range(9)), [1.0] * 9), ([1.0, 2.0], [1.0])):
        with pytest.raises(ValueError):
            s.set_mass_table("phi", times, masses)


def test_mass_table_marshalled_into_the_config():
    """The knots reach best_species as the header lays them out (ctypes
    only, no library call)."""
    from paper_2603_28848_gb300 import config_from_problem
    s = Solver(0.1, 20.0, 8)
    s.initialize_species("A", lambda q: np.exp(-q), stat="maxwell", mass=0.3, mass_slope=0.2)
    s.initialize_species("B", lambda q: np.exp(-q), stat="boson")
    s.set_mass_table("B", [0.5, 1.5, 3.0], [2.0, 1.0, 0.0])
    s.add_process("AB", ["A", "B"], ["A", "B"], neval=100)
    cfg, keep = config_from_problem(s.problem(), W.PREC_FP64)
    a, b = cfg.species[0], cfg.species[1]
    assert a.n_mass_knots == 0 and a.mass0 == 0.3 and a.mass1 == 0.2
    assert b.n_mass_knots == 3 and list(b.mass_t[:3]) == [0.5, 1.5, 3.0] and list(b.mass_m[:3]) == [2.0, 1.0, 0.0]
