"""VEGAS adaptive map, training data, refinement and iteration combination.

Test infrastructure (see ``oracle/__init__``).

The paper integrates with the ``vegas`` library (Sec. 3A) and names its
parameters neval, nitn and alpha (Sec. 3A, App. C: alpha = 0.5, nitn = 2) and
the reuse of the adapted map across grid points and time steps (Sec. 3D).
The map and its refinement here follow Lepage's published algorithm
(G. P. Lepage, J. Comput. Phys. 27 (1978) 192; J. Comput. Phys. 439 (2021)
110386), without the adaptive stratification of the library's default:

  * each dimension has nb increments with edges 0 = e_0 < ... < e_nb = 1;
    a uniform x in (0,1) falls in increment b = floor(x nb) (clamped to
    nb-1) and maps to y = e_b + (e_{b+1} - e_b)(x nb - b) with Jacobian
    nb (e_{b+1} - e_b); the sample weight is the integrand times the product
    of the per-dimension Jacobians;
  * training data: d_b = sum of squared sample weights over samples whose x
    falls in increment b (per dimension);
  * refinement: smooth d with the (7,1)/8, (1,6,1)/8, (1,7)/8 stencil,
    normalise to unit sum, compress with ((1 - d)/ln(1/d))^alpha (zero where
    d = 0), then choose new edges so that each new increment holds an equal
    share of the compressed weight, interpolating linearly inside old
    increments.  A dimension whose d is all zero keeps its edges.

Reading (not in the paper or in Lepage's description): a smoothed,
normalised share below EMPTY_SHARE = 1e-30 counts as an empty increment
(compressed weight 0, like d = 0).  The compression jumps from about 0.1 for
a tiny positive share to 0 for an exact zero, so without this rule the map
would depend on where floating-point underflow of w^2 falls, i.e. on the
overall scale of w and on the precision of the training data.
"""
import numpy as np

EMPTY_SHARE = 1e-30


def uniform_edges(dim, nbins):
    """Initial map: nb equal increments per dimension, shape (dim, nbins+1)."""
    return np.tile(np.linspace(0.0, 1.0, nbins + 1), (dim, 1))


def apply_map(edges, x):
    """Map uniforms x (N, D) to y (N, D); returns (y, jac (N,), bins (N, D))."""
    nb = edges.shape[1] - 1
    t = x * nb
    b = np.minimum(np.floor(t).astype(np.int64), nb - 1)
    frac = t - b
    d_idx = np.arange(edges.shape[0])[None, :]
    lo = edges[d_idx, b]
    width = edges[d_idx, b + 1] - lo
    y = lo + width * frac
    jac = np.prod(nb * width, axis=1)
    return y, jac, b


def training_data(bins, w, nbins):
    """d[dim, b] = sum of w^2 over samples with x in increment b of dim."""
    w2 = w * w
    return np.stack([np.bincount(bins[:, k], weights=w2, minlength=nbins)
                     for k in range(bins.shape[1])])


def refine_1d(edges, d, alpha):
    """One refinement of a single dimension's edges from its training data."""
    nb = len(d)
    d = np.asarray(d, dtype=np.float64)
    if not np.any(d > 0):
        return edges.copy()
    # smoothing with nearest neighbours
    s = np.empty(nb)
    if nb == 1:
        s[0] = d[0]
    else:
        s[0] = (7.0 * d[0] + d[1]) / 8.0
        s[-1] = (d[-2] + 7.0 * d[-1]) / 8.0
        s[1:-1] = (d[:-2] + 6.0 * d[1:-1] + d[2:]) / 8.0
    s = s / s.sum()
    # compression (damping) with exponent alpha
    omega = np.zeros(nb)
    for b in range(nb):
        if s[b] < EMPTY_SHARE:
            omega[b] = 0.0
        elif s[b] >= 1.0:
            omega[b] = 1.0
        else:
            omega[b] = ((1.0 - s[b]) / -np.log(s[b])) ** alpha
    # re-partition into nb increments of equal compressed weight
    target = omega.sum() / nb
    new = np.empty(nb + 1)
    new[0] = 0.0
    new[nb] = 1.0
    acc = 0.0          # compressed weight of old increments before index i
    i = 0
    for k in range(1, nb):
        goal = k * target
        while i < nb - 1 and acc + omega[i] < goal:
            acc += omega[i]
            i += 1
        frac = (goal - acc) / omega[i] if omega[i] > 0.0 else 0.0
        new[k] = edges[i] + min(max(frac, 0.0), 1.0) * (edges[i + 1] - edges[i])
    return new


def refine(edges, d, alpha):
    """Refine every dimension of a map; edges (D, nb+1), d (D, nb)."""
    return np.stack([refine_1d(edges[k], d[k], alpha) for k in range(edges.shape[0])])


def iteration_estimate(sum_w, sum_w2, n):
    """Mean and variance of the mean from one iteration's sums."""
    mean = sum_w / n
    var = (sum_w2 / n - mean * mean) / (n - 1) if n > 1 else 0.0
    return mean, max(var, 0.0)


def combine(means, variances):
    """Inverse-variance weighted mean of the iterations and its standard error.

    Reading: iterations with zero variance (an integrand that vanished on all
    samples) are exact; if any exist, their plain mean is returned with zero
    error.
    """
    means = np.asarray(means, dtype=np.float64)
    variances = np.asarray(variances, dtype=np.float64)
    exact = variances <= 0.0
    if np.any(exact):
        return float(np.mean(means[exact])), 0.0
    wts = 1.0 / variances
    mean = float(np.sum(wts * means) / np.sum(wts))
    return mean, float(np.sqrt(1.0 / np.sum(wts)))
