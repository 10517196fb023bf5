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


def _s_of(momenta, n_in=2):
    tot = momenta[:n_in].sum(axis=0)
    return tot[0] ** 2 - tot[1] ** 2 - tot[2] ** 2 - tot[3] ** 2


def test_matrix_element_callable_reduced_to_p_of_s():
    """A callable |M|^2(momenta, coupling) that is a cubic in the initial
    state's s is reduced to its coefficients; a constant one to (1, 0, 0, 0)."""
    from paper_2603_28848_gb300.solver import matrix_element_polynomial
    const = matrix_element_polynomial(lambda k, g: g * g * np.ones(k.shape[2]), 0.7, [1.0, 1.0], [1.0, 1.0], 20.0)
    assert np.allclose(const, (1.0, 0.0, 0.0, 0.0), rtol=0, atol=1e-12)
    want = (0.5, 0.3, 0.05, 0.002)
    fn = lambda k, g: g ** 2 * (want[0] + want[1] * _s_of(k) + want[2] * _s_of(k) ** 2 + want[3] * _s_of(k) ** 3)
    got = matrix_element_polynomial(fn, 1.3, [0.5, 0.8], [0.5, 0.8, 0.1], 10.0)
    assert np.allclose(got, want, rtol=1e-7, atol=0)
    # the same through the solver, with the paper's argument order
    s = Solver(0.1, 10.0, 8)
    s.initialize_species("A", lambda q: np.exp(-q), stat="maxwell", mass=0.5)
    s.initialize_species("B", lambda q: np.exp(-q), stat="maxwell", mass=0.8)
    s.add_process("AB", ["A", "B"], ["A", "B"], fn, coupling=1.3, neval=100)
    s.add_process("AB2", ["A", "B"], ["A", "B"], (2.0, 0.1), coupling=1.0, neval=100)
    p = s.problem().processes
    assert np.allclose(p[0].me_coef, want, rtol=1e-7) and p[1].me_coef == (2.0, 0.1, 0.0, 0.0)
    with pytest.raises(ValueError):
        s.add_process("both", ["A", "B"], ["A", "B"], fn, me_coef=(1.0,))


def test_matrix_element_not_a_cubic_in_s_is_refused():
    """Dependence on a final momentum (a t-channel invariant), a quartic in s
    and a zero coupling cannot be represented and raise."""
    from paper_2603_28848_gb300.solver import matrix_element_polynomial

    def t_channel(k, g):
        d = k[0] - k[2]
        return g * g * (1.0 + 0.1 * (d[0] ** 2 - d[1] ** 2 - d[2] ** 2 - d[3] ** 2))

    with pytest.raises(ValueError):
        matrix_element_polynomial(t_channel, 1.0, [1.0, 1.0], [1.0, 1.0], 20.0)
    with pytest.raises(ValueError):
        matrix_element_polynomial(lambda k, g: g * g * _s_of(k) ** 4, 1.0, [1.0, 1.0], [1.0, 1.0], 20.0)
    with pytest.raises(ValueError):
        matrix_element_polynomial(lambda k, g: np.ones(k.shape[2]), 0.0, [1.0, 1.0], [1.0, 1.0], 20.0)
