"""Pins of the oracle's VEGAS map, refinement and iteration combination."""
import numpy as np
import pytest

from oracle import philox, vegas


def _random_map(rng, D, nb):
    w = rng.uniform(0.1, 3.0, size=(D, nb))
    e = np.concatenate([np.zeros((D, 1)), np.cumsum(w, axis=1)], axis=1)
    return e / e[:, -1:]


def test_uniform_map_is_identity():
    e = vegas.uniform_edges(3, 50)
    x = np.random.default_rng(0).uniform(size=(1000, 3))
    y, jac, b = vegas.apply_map(e, x)
    assert np.allclose(y, x, atol=1e-15)
    assert np.allclose(jac, 1.0)


def test_jacobian_integrates_to_one_exactly():
    """Int_0^1 J(x) dx = sum of increment widths = 1 for any map: one
    midpoint sample per increment integrates the piecewise-constant J exactly."""
    rng = np.random.default_rng(1)
    e = _random_map(rng, 1, 50)
    x = ((np.arange(50) + 0.5) / 50)[:, None]
    y, jac, b = vegas.apply_map(e, x)
    assert np.isclose(np.mean(jac), 1.0, rtol=1e-14)
    assert np.array_equal(b[:, 0], np.arange(50))


def test_map_is_monotone_and_continuous():
    rng = np.random.default_rng(2)
    e = _random_map(rng, 2, 20)
    x = np.linspace(1e-9, 1 - 1e-9, 20001)[:, None].repeat(2, axis=1)
    y, _, _ = vegas.apply_map(e, x)
    assert np.all(np.diff(y, axis=0) > 0)
    assert np.max(np.diff(y, axis=0)) < 1e-3     # no jumps at increment edges


def test_refine_concentrated_weight_by_hand():
    """All training weight in increment 2 of 4, alpha = 1: smoothing gives
    (0, 1, 6, 1)/8; compression gives omega_b = (1 - s)/ln(1/s); equal shares
    of sum(omega)/4 are then read off the cumulative weight by hand."""
    e = np.linspace(0, 1, 5)
    d = np.array([0.0, 0.0, 1.0, 0.0])
    new = vegas.refine_1d(e, d, 1.0)
    s = np.array([0.0, 1.0, 6.0, 1.0]) / 8.0
    om = np.array([0.0] + [(1 - v) / np.log(1 / v) for v in s[1:]])
    tot = om.sum()
    cum = np.concatenate([[0.0], np.cumsum(om)])
    want = [0.0]
    for k in (1, 2, 3):
        g = k * tot / 4
        i = np.searchsorted(cum, g) - 1
        want.append(0.25 * i + 0.25 * (g - cum[i]) / om[i])
    want.append(1.0)
    assert np.allclose(new, want, rtol=0, atol=1e-14)
    # the weighted increment ends up narrower than its neighbours' share
    assert new[3] - new[2] < 0.25


def test_refine_keeps_uniform_data_fixed_and_zero_data_unchanged():
    e = vegas.uniform_edges(1, 10)[0]
    assert np.allclose(vegas.refine_1d(e, np.ones(10), 0.5), e, atol=1e-14)
    rng = np.random.default_rng(3)
    e2 = _random_map(rng, 1, 10)[0]
    assert np.array_equal(vegas.refine_1d(e2, np.zeros(10), 0.5), e2)


def _gauss_integrand(y, c=0.4, s=0.08):
    return np.prod(np.exp(-(y - c) ** 2 / (2 * s * s)) / (s * np.sqrt(2 * np.pi)), axis=1)


def _run(D, nitn, N, seed, alpha=0.5, nb=50):
    from scipy.special import erf
    e = vegas.uniform_edges(D, nb)
    its = []
    for it in range(nitn):
        x = philox.uniforms(seed, 0, it, 0, N, D, "f64")
        y, jac, b = vegas.apply_map(e, x)
        w = _gauss_integrand(y) * jac
        its.append(vegas.iteration_estimate(w.sum(), (w * w).sum(), N))
        e = vegas.refine(e, vegas.training_data(b, w, nb), alpha)
    one = 0.5 * (erf((1 - 0.4) / (0.08 * np.sqrt(2))) - erf((0 - 0.4) / (0.08 * np.sqrt(2))))
    exact = one ** D
    return its, vegas.combine([m for m, _ in its], [v for _, v in its]), exact


@pytest.mark.parametrize("D", [6, 12])
def test_known_integral_and_adaptation(D):
    """Product of 1-D Gaussians: the combined estimate lies within 3 sigma of
    the exact value and the map adaptation shrinks the per-iteration error."""
    its, (mean, err), exact = _run(D, 6, 20_000, 17)
    assert abs(mean - exact) < 3 * err + 1e-12
    assert np.sqrt(its[-1][1]) < 0.2 * np.sqrt(its[0][1])


def test_error_estimate_coverage():
    """Over independent seeds the reported standard error matches the scatter:
    the z-scores have unit variance and about 68% fall within one sigma."""
    z = []
    for seed in range(40):
        its, (mean, err), exact = _run(2, 3, 4000, 1000 + seed)
        z.append((mean - exact) / err)
    z = np.array(z)
    assert 0.6 < np.std(z) < 1.5
    assert abs(np.mean(z)) < 0.6


def test_combine_inverse_variance():
    """Two estimates with variances 1 and 4: the weighted mean is 4/5 of the
    way to the more precise one and the combined variance is 4/5."""
    m, e = vegas.combine([1.0, 6.0], [1.0, 4.0])
    assert np.isclose(m, 2.0) and np.isclose(e * e, 0.8)
    m, e = vegas.combine([0.0, 0.0], [0.0, 0.0])
    assert m == 0.0 and e == 0.0


def test_refine_is_scale_invariant():
    """Training data that differ by a constant factor give the same map,
    even when the factor moves w^2 across the floating-point underflow
    threshold (the empty-share reading)."""
    rng = np.random.default_rng(5)
    e = vegas.uniform_edges(1, 50)[0]
    x = rng.uniform(size=4000)
    w = np.exp(-((x - 0.37) / 0.004) ** 2 / 2)          # a narrow peak: most w^2 underflow
    b = np.minimum((x * 50).astype(int), 49)
    ref = None
    for sc in (1.0, 1e-5, 1e5, 1e20, 1e-20):
        d = np.bincount(b, weights=(sc * w) ** 2, minlength=50)
        new = vegas.refine_1d(e, d, 0.5)
        if ref is None:
            ref = new
        assert np.max(np.abs(new - ref)) < 1e-12
