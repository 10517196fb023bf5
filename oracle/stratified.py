"""Adaptive stratified sampling on top of the VEGAS map (VEGAS+).

Test infrastructure (see ``oracle/__init__``).

The paper integrates with the ``vegas`` library, whose default since 2021
combines the adaptive map with adaptive stratified sampling (G. P. Lepage,
J. Comput. Phys. 439 (2021) 110386): the unit cube of the map's input is cut
into H = M^D equal hypercubes, each gets its own number of samples, drawn
uniformly inside it, and after every iteration the samples are redistributed
in proportion to a damped power of each hypercube's standard deviation.  The
iteration estimate is the sum of the hypercubes' sample means times their
volume 1/H, and its variance the sum of their variances of the mean times
1/H^2.

Readings (the paper says nothing about the stratification; the library's
internals are not restated here, only the published method):
  * samples come in items of C = 8 consecutive samples of the task's stream
    (sample k is in item k // C); a task draws J = floor(N / C) items, so
    C J samples; an item lies in one hypercube, and the items of a
    hypercube are consecutive, in hypercube order;
  * M is the largest integer >= 1 with 4 M^D <= J and M^D <= H_max (at
    least four items per hypercube on average); hypercube
    h = sum_d i_d M^d (dimension 0 fastest), x_d = (i_d + u_d) / M with u the
    sample's uniforms;
  * allocation m_h >= 1 items with sum m_h = J; the first iteration of a task
    is uniform, m_h = floor(J / H) + [h < J mod H];
  * with n_h = C m_h, S1_h = sum w, S2_h = sum w^2 over the hypercube's
    samples: I = (1/H) sum_h S1_h / n_h and
    Var = (1/H^2) sum_h s_h^2 / n_h, s_h^2 = max(0, (S2_h - S1_h^2 / n_h) / (n_h - 1));
  * the map's training data weight each sample by the volume it stands for:
    d_b = sum over samples in increment b of w^2 / m_h;
  * the next allocation: d_h = (s_h^2)^(beta/2) (beta = 0.75 damps it);
    m_h = 1 + floor((J - H) d_h / sum d), the J - sum m_h items left over go
    one each to h = 0, 1, ...; if every d_h is 0 (or rounding made
    sum m_h exceed J) the allocation is uniform;
  * map refinement and reallocation both use the same iteration's samples;
    the allocation persists across evaluations like the map.
"""
import numpy as np

CHUNK_ITEMS = 8          # C: samples per item


def shape(n_samples, dim, max_hcubes):
    """(M, H, J): strata per dimension, hypercubes and items of a task; M is
    the largest integer >= 1 with 4 M^D <= J and M^D <= max_hcubes (integer
    comparisons, so no rounding of a root is involved)."""
    J = n_samples // CHUNK_ITEMS
    if J < 1:
        raise ValueError("stratified sampling needs at least one item of 8 samples")
    M = 1
    while 4 * (M + 1) ** dim <= J and (M + 1) ** dim <= max_hcubes:
        M += 1
    return M, M ** dim, J


def uniform_allocation(J, H):
    m = np.full(H, J // H, dtype=np.int64)
    m[: J % H] += 1
    return m


def digits(h, M, dim):
    """Stratum index i_d of hypercubes h (array) per dimension, shape (len(h), dim)."""
    h = np.asarray(h, dtype=np.int64)
    out = np.empty((h.size, dim), dtype=np.int64)
    r = h.copy()
    for d in range(dim):
        out[:, d] = r % M
        r //= M
    return out


def estimate(S1, S2, m):
    """Iteration estimate and variance of the mean from per-hypercube sums."""
    H = len(m)
    n = CHUNK_ITEMS * np.asarray(m, dtype=np.float64)
    s2 = np.maximum((S2 - S1 * S1 / n) / (n - 1.0), 0.0)
    mean = np.sum(S1 / n) / H
    var = np.sum(s2 / n) / (H * H)
    return float(mean), float(var), s2


def allocate(s2, J, beta):
    """Items per hypercube for the next iteration from the sample variances."""
    H = len(s2)
    d = np.power(s2, 0.5 * beta)
    tot = np.sum(d)
    if not tot > 0.0:
        return uniform_allocation(J, H)
    m = 1 + np.floor((J - H) * d / tot).astype(np.int64)
    rest = J - int(np.sum(m))
    if rest < 0:                       # rounding overshoot: start afresh
        return uniform_allocation(J, H)
    m[:rest] += 1
    return m
