"""Pins of the oracle's time-dependent mass (Sec. 3A): the linear law and the
piecewise-linear knot table, checked against values worked out by hand."""
import numpy as np
import pytest

from oracle.collision import mass_of, masses
from workloads import STAT_BE, Grid, Problem, Process, Species


def test_linear_law():
    sp = Species("phi", STAT_BE, 0.5, 0.25)
    assert mass_of(sp, 0.0) == 0.5
    assert mass_of(sp, 2.0) == 1.0
    assert mass_of(sp, -2.0) == 0.0


def test_table_by_hand():
    """Knots (1, 2), (2, 1), (4, 0): the knots themselves, the midpoints
    (1.5 and 0.5), a quarter of the way (t = 2.5 -> 0.75) and the constant
    continuation beyond either end."""
    sp = Species("phi", STAT_BE, 9.0, 9.0, ((1.0, 2.0), (2.0, 1.0), (4.0, 0.0)))
    want = {0.0: 2.0, 1.0: 2.0, 1.5: 1.5, 2.0: 1.0, 2.5: 0.75, 3.0: 0.5, 4.0: 0.0, 7.0: 0.0}
    for t, m in want.items():
        assert mass_of(sp, t) == pytest.approx(m, rel=0, abs=1e-15), t


def test_table_through_a_line_is_the_line():
    """Knots placed on m = 0.3 + 0.2 t reproduce the linear law anywhere
    between them; a two-knot table is the straight line through them."""
    lin = Species("a", STAT_BE, 0.3, 0.2)
    tk = [0.0, 0.7, 1.1, 3.0, 5.5]
    tab = Species("b", STAT_BE, 0.0, 0.0, tuple((t, 0.3 + 0.2 * t) for t in tk))
    for t in np.linspace(0.0, 5.5, 37):
        assert mass_of(tab, t) == pytest.approx(mass_of(lin, t), rel=1e-14)
    two = Species("c", STAT_BE, 0.0, 0.0, ((2.0, 1.0), (6.0, 3.0)))
    assert mass_of(two, 5.0) == pytest.approx(2.5, rel=1e-15)


def test_table_is_continuous_and_monotone_per_segment():
    """Near each interior knot the interpolant approaches the knot's mass
    from both sides, and between knots it stays between their masses."""
    tab = ((0.5, 1.0), (1.0, 0.1), (1.2, 0.1), (3.0, 2.0))
    sp = Species("phi", STAT_BE, 0.0, 0.0, tab)
    for (ta, ma), (tb, mb) in zip(tab[:-1], tab[1:]):
        for t in np.linspace(ta, tb, 11):
            assert min(ma, mb) - 1e-15 <= mass_of(sp, t) <= max(ma, mb) + 1e-15
        assert abs(mass_of(sp, tb - 1e-9) - mb) < 1e-7 * (1 + abs(mb - ma) / (tb - ta))
        assert abs(mass_of(sp, ta + 1e-9) - ma) < 1e-7 * (1 + abs(mb - ma) / (tb - ta))


def test_masses_per_species_and_list_knots():
    """masses() takes each species' own law; knots given as lists (as a JSON
    checkpoint returns them) become the same table."""
    a = Species("a", STAT_BE, 1.0)
    b = Species("b", STAT_BE, 0.0, 0.0, [[0.0, 0.0], [2.0, 4.0]])
    assert b.mass_table == ((0.0, 0.0), (2.0, 4.0))
    prob = Problem(Grid(4, 0.1, 1.0), (a, b), (Process("ab", (0, 1), (0, 1)),))
    assert np.array_equal(masses(prob, 1.0), [1.0, 2.0])


def test_table_equals_library_interpolation():
    """Random tables against numpy's piecewise-linear interpolation (which
    also holds the end values outside the knots)."""
    rng = np.random.default_rng(7)
    for _ in range(50):
        k = int(rng.integers(2, 9))
        tk = np.cumsum(rng.uniform(0.01, 2.0, k)) - 1.0
        mk = rng.uniform(0.0, 3.0, k)
        sp = Species("phi", STAT_BE, 0.0, 0.0, tuple(zip(tk, mk)))
        for t in rng.uniform(tk[0] - 1.0, tk[-1] + 1.0, 20):
            assert mass_of(sp, t) == pytest.approx(np.interp(t, tk, mk), rel=1e-13, abs=1e-15)
