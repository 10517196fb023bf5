"""Independent exact-energy reductions of the 2 -> 2 collision integral.

Test infrastructure (see ``oracle/__init__``).  These are the pins of the
Monte Carlo oracle: each reduces the same single-position integral of
Eq. (3) with the exact delta function (no Gaussian), by a route that shares
nothing with the Monte Carlo kinematics.

  * ``loss_massless_mb``: closed form for massless MB legs and constant
    |M|^2 without momentum cuts.  With the two-body phase space
    Int dPhi_2 = 1/(8 pi) and Int d^3p/((2pi)^3 2p) A e^{-p/T} = A T^2/(4 pi^2):
        loss(p1) = lambda^2 A^2 T^2 exp(-p1/T) / (64 pi^3 p1).
  * ``two_body_cm``: the centre-of-mass reduction for general masses and
    statistics: integrate d^3p2 in the lab (p2, cos theta_2; the azimuth gives
    2 pi), and the two-body phase space of (p3, p4) in the centre-of-mass
    frame, dPhi_2 = |p*| / (16 pi^2 sqrt(s)) dOmega*, with the polar axis
    along the total momentum so that the lab energies depend only on
    cos theta* (the azimuth gives 2 pi).  Gauss-Legendre quadrature in
    (p2, cos theta_2, cos theta*).
  * ``paper_backward_term``: the paper's own semi-analytic backward term
    C_BW of Eq. (18)-(19) with the kinematic function F of App. B, taken as
    printed.
"""
import numpy as np

TWO_PI = 2.0 * np.pi


def loss_massless_mb(p1, A, T, lam=1.0):
    """Closed-form single-position loss term for massless MB 2 -> 2."""
    return lam ** 2 * A ** 2 * T ** 2 * np.exp(-p1 / T) / (64.0 * np.pi ** 3 * p1)


def _gl(a, b, n):
    x, w = np.polynomial.legendre.leggauss(n)
    return 0.5 * (b - a) * x + 0.5 * (b + a), 0.5 * (b - a) * w


def composite_gl(breaks, n):
    xs, ws = [], []
    for a, b in zip(breaks[:-1], breaks[1:]):
        x, w = _gl(a, b, n)
        xs.append(x)
        ws.append(w)
    return np.concatenate(xs), np.concatenate(ws)


def two_body_cm(p1, masses, f1, dist2, dist3, dist4, eta, lam=1.0, term="loss",
                r_cut=None, p2_breaks=(0, 0.25, 0.5, 1, 2, 4, 8, 16, 32, 64),
                n_p2=24, n_c2=48, n_cs=48, omega=0.0, me=None):
    """Single-position 2 -> 2 gain or loss term at observed momentum p1.

    Legs: 1 = observed (initial side), 2 = other initial leg, 3 and 4 = final
    legs; ``dist_k(q)`` give f_k, ``eta`` = (eta1..eta4) the (1 + eta f)
    signs; ``r_cut`` = (q_min, q_max) restricts |p3| and |p4| as the Monte
    Carlo restricts its integrated legs.  ``omega`` shifts the energy
    balance to E3 + E4 = E1 + E2 - omega (used by ``two_body_cm_smeared``);
    a callable omega(E_in) returns (omega, weight) arrays for the initial
    energy E_in = E1 + E2 of each node, the weight multiplying the integrand
    (used by ``two_body_cm_fractional``).  ``me(s)`` multiplies |M|^2 = lam^2 by
    a function of the initial state's invariant mass squared s = (E1 + E2)^2 -
    |p1 + p2|^2 (constant when None).
    """
    m1, m2, m3, m4 = masses
    e1, e2, e3, e4 = eta
    E1 = np.sqrt(p1 * p1 + m1 * m1)
    p2, w2 = composite_gl(p2_breaks, n_p2)
    c2, wc2 = _gl(-1.0, 1.0, n_c2)
    cs, wcs = _gl(-1.0, 1.0, n_cs)
    P2, C2, CS = np.meshgrid(p2, c2, cs, indexing="ij")
    W = w2[:, None, None] * wc2[None, :, None] * wcs[None, None, :]
    E2 = np.sqrt(P2 ** 2 + m2 * m2)
    extra = 1.0
    if callable(omega):
        omega, extra = omega(E1 + E2)
    Ptot = np.sqrt(np.maximum(p1 * p1 + P2 ** 2 + 2.0 * p1 * P2 * C2, 0.0))
    Etot = E1 + E2 - omega
    s = Etot ** 2 - Ptot ** 2
    ok = (s > (m3 + m4) ** 2) & (Etot > 0.0)
    s = np.where(ok, s, (m3 + m4) ** 2 + 1.0)
    rs = np.sqrt(s)
    pstar = np.sqrt((s - (m3 + m4) ** 2) * (s - (m3 - m4) ** 2)) / (2.0 * rs)
    E3s = (s + m3 * m3 - m4 * m4) / (2.0 * rs)
    beta = Ptot / Etot
    gamma = Etot / rs
    E3 = gamma * (E3s + beta * pstar * CS)
    E4 = Etot - E3
    q3 = np.sqrt(np.maximum(E3 ** 2 - m3 * m3, 0.0))
    q4 = np.sqrt(np.maximum(E4 ** 2 - m4 * m4, 0.0))
    f2 = dist2(P2)
    f3 = dist3(q3)
    f4 = dist4(q4)
    if term == "gain":
        stat = f3 * f4 * (1.0 + e1 * f1) * (1.0 + e2 * f2)
    else:
        stat = f1 * f2 * (1.0 + e3 * f3) * (1.0 + e4 * f4)
    keep = ok.copy()
    if r_cut is not None:
        lo, hi = r_cut
        keep &= (q3 >= lo) & (q3 <= hi) & (q4 >= lo) & (q4 <= hi)
    # dPhi_2 integrated over the azimuth phi*: 2 pi |p*| / (16 pi^2 sqrt(s))
    phase = TWO_PI * pstar / (16.0 * np.pi ** 2 * rs)
    # d^3p2 / ((2pi)^3 2E2) with the azimuth of p2 giving 2 pi
    meas = TWO_PI * P2 ** 2 / (TWO_PI ** 3 * 2.0 * E2)
    if me is not None:
        sin_ = (E1 + E2) ** 2 - Ptot ** 2          # initial state, before the omega shift
        extra = extra * me(sin_)
    val = lam ** 2 * stat * phase * meas / (2.0 * E1) * extra
    return float(np.sum(np.where(keep, val, 0.0) * W))


def two_body_cm_smeared(p1, masses, f1, dist2, dist3, dist4, eta, sigma, lam=1.0,
                        term="loss", r_cut=None, n_omega=32, width=7.0, **kw):
    """The same term with the delta of energy replaced by the Gaussian of
    Eq. (11): Int d omega G_sigma(omega) X(omega), X the exact-delta term at
    energy imbalance E_in - E_out = omega (Gauss-Legendre in omega)."""
    om, wom = _gl(-width * sigma, width * sigma, n_omega)
    g = np.exp(-om ** 2 / (2.0 * sigma ** 2)) / (sigma * np.sqrt(TWO_PI))
    return float(sum(wk * gk * two_body_cm(p1, masses, f1, dist2, dist3, dist4, eta, lam,
                                           term, r_cut, omega=o, **kw)
                     for o, wk, gk in zip(om, wom, g)))


def two_body_cm_fractional(p1, masses, f1, dist2, dist3, dist4, eta, w, lam=1.0,
                           term="loss", r_cut=None, n_z=32, width=7.0, **kw):
    """The same term with the fractional width of App. C: the Gaussian in
    omega = E_in - E_out has sigma = w (E_in + E_out) / 2 = w (2 E_in - omega) / 2.
    With omega = z sigma this gives omega = z w E_in / (1 + z w / 2) and
    G d omega = phi(z) dz / (1 + z w / 2), phi the unit normal density;
    Gauss-Legendre in z over [-width, width]."""
    z, wz = _gl(-width, width, n_z)
    total = 0.0
    for zk, wk in zip(z, wz):
        den = 1.0 + 0.5 * zk * w
        phi = np.exp(-0.5 * zk * zk) / np.sqrt(TWO_PI)
        om = lambda E_in, zk=zk, den=den: (zk * w * E_in / den, 1.0 / den)
        total += wk * phi * two_body_cm(p1, masses, f1, dist2, dist3, dist4, eta, lam, term, r_cut,
                                        omega=om, **kw)
    return float(total)


def paper_backward_term(p1, masses, f1, dist2, dist3, dist4, eta, lam=1.0,
                        p_breaks=(0, 0.25, 0.5, 1, 2, 4, 8, 16, 32), n_p=24, n_c=96):
    """C_BW(p1) of Eq. (18) with F of App. B, as printed (exact energy).

    E2 = E3 + E4 - E1 and p2 = sqrt(E2^2 - m2^2); F integrates
    |M|^2 pi / sqrt(-a) over cos(theta) where b^2 - 4ac >= 0, with
    Q, gamma, eps, kappa, a, b, c as in App. B.
    """
    m1, m2, m3, m4 = masses
    e1, e2, e3, e4 = eta
    E1 = np.sqrt(p1 * p1 + m1 * m1)
    p3, w3 = composite_gl(p_breaks, n_p)
    p4, w4 = composite_gl(p_breaks, n_p)
    ct, wct = _gl(-1.0, 1.0, n_c)
    P3, P4, CT = np.meshgrid(p3, p4, ct, indexing="ij")
    E3 = np.sqrt(P3 ** 2 + m3 * m3)
    E4 = np.sqrt(P4 ** 2 + m4 * m4)
    E2 = E3 + E4 - E1
    okE = E2 > m2
    p2 = np.sqrt(np.maximum(E2 ** 2 - m2 * m2, 0.0))
    Q = m1 ** 2 - m2 ** 2 + m3 ** 2 + m4 ** 2
    gam = E3 * E4 - E1 * E3 - E1 * E4
    eps = p1 * P3 * CT
    kap = p1 ** 2 + P3 ** 2
    a = P4 ** 2 * (-4.0 * kap + 8.0 * eps)
    b = P4 * (-p1 + eps / p1) * (8.0 * gam + 4.0 * Q + 8.0 * eps)
    sin2 = 1.0 - CT ** 2
    c = 4.0 * P3 ** 2 * P4 ** 2 * sin2 - (2.0 * (gam + eps) + Q) ** 2
    okF = (b * b - 4.0 * a * c >= 0.0) & (a < 0.0)
    F_int = np.where(okF, lam ** 2 * np.pi / np.sqrt(np.where(a < 0.0, -a, 1.0)), 0.0)
    F = np.sum(F_int * wct[None, None, :], axis=2)
    okE2 = okE[:, :, 0]
    f2 = dist2(p2[:, :, 0])
    f3 = dist3(P3[:, :, 0])
    f4 = dist4(P4[:, :, 0])
    stat = f3 * f4 * (1.0 + e1 * f1) * (1.0 + e2 * f2)
    integ = (P3[:, :, 0] ** 2 / (2.0 * E3[:, :, 0])) * (P4[:, :, 0] ** 2 / (2.0 * E4[:, :, 0])) * F * stat
    integ = np.where(okE2, integ, 0.0)
    W = w3[:, None] * w4[None, :]
    return float(2.0 / TWO_PI ** 4 / (2.0 * E1) * np.sum(integ * W))


# ----------------------------------------------------------------------------
# 2 <-> 3 with MB legs of equal mass m and constant |M|^2 (pins of the
# five-leg side integrals C_2 and C_3 of Sec. 2C).
# ----------------------------------------------------------------------------

def phase2(s, m):
    """Two-body phase space of equal masses: sqrt(1 - 4m^2/s) / (8 pi)."""
    s = np.asarray(s, dtype=np.float64)
    x = np.where(s > 4 * m * m, 1.0 - 4 * m * m / np.where(s > 0, s, 1.0), 0.0)
    return np.sqrt(x) / (8.0 * np.pi)


def phase3(s, m, n=48):
    """Three-body phase space of equal masses from the Dalitz-plot area:
    Phi_3 = Area / (128 pi^3 s), Area = Int dm12^2 (m23^2_max - m23^2_min)."""
    s = np.atleast_1d(np.asarray(s, dtype=np.float64))
    out = np.zeros_like(s)
    ok = s > 9 * m * m
    rs = np.sqrt(s[ok])
    lo = 4 * m * m
    hi = (rs - m) ** 2
    xg, wg = np.polynomial.legendre.leggauss(n)
    x = 0.5 * (hi - lo)[:, None] * xg[None, :] + 0.5 * (hi + lo)[:, None]
    w = 0.5 * (hi - lo)[:, None] * wg[None, :]
    rx = np.sqrt(x)
    e2 = rx / 2.0
    e3 = (s[ok][:, None] - x - m * m) / (2.0 * rx)
    width = 4.0 * np.sqrt(np.maximum(e2 * e2 - m * m, 0)) * np.sqrt(np.maximum(e3 * e3 - m * m, 0))
    out[ok] = np.sum(width * w, axis=1) / (128.0 * np.pi ** 3 * s[ok])
    return out


def loss_2to3_c2_mb(p0, m, A, T, sigma, lam=1.0, n_p=32, n_c=32, n_om=24,
                    p_breaks=(0, 0.5, 1, 2, 4, 8, 16, 32)):
    """Loss of C_2 (observed on the 2-leg side) for MB legs f = A e^{-E/T}
    with the Gaussian of Eq. (11): f0/(2E0) Int d^3p1/((2pi)^3 2E1) f1 |M|^2
    Int d omega G(omega) Phi_3((E0+E1-omega)^2 - |p0+p1|^2)."""
    E0 = np.sqrt(p0 * p0 + m * m)
    p1, w1 = composite_gl(p_breaks, n_p)
    c, wc = _gl(-1.0, 1.0, n_c)
    om, wom = _gl(-7 * sigma, 7 * sigma, n_om)
    P1, C, OM = np.meshgrid(p1, c, om, indexing="ij")
    W = w1[:, None, None] * wc[None, :, None] * wom[None, None, :]
    E1 = np.sqrt(P1 ** 2 + m * m)
    Pt2 = p0 * p0 + P1 ** 2 + 2 * p0 * P1 * C
    Ef = E0 + E1 - OM
    s = np.where(Ef > 0, Ef ** 2 - Pt2, 0.0)
    ph = phase3(s.reshape(-1), m).reshape(s.shape)
    g = np.exp(-OM ** 2 / (2 * sigma ** 2)) / (sigma * np.sqrt(TWO_PI))
    f0 = A * np.exp(-E0 / T)
    f1 = A * np.exp(-E1 / T)
    meas = TWO_PI * P1 ** 2 / (TWO_PI ** 3 * 2 * E1)
    return float(lam ** 2 * f0 / (2 * E0) * np.sum(meas * f1 * g * ph * W))


def loss_2to3_c3_mb(p2, m, A, T, sigma, lam=1.0, n_e=40, n_k=32, n_c=24, n_om=20):
    """Loss of C_3 (observed on the 3-leg side) for MB legs: the two other
    final legs enter only through K = p3 + p4 and f3 f4 = A^2 e^{-K0/T}, so
    loss = f2 A^2 / (2E2 (2pi)^4) Int d^4K e^{-K0/T} Phi_2(K^2)
           Int d omega G(omega) Phi_2((E2 + K0 + omega)^2 - |p2 + K|^2),
    with d^4K = dK0 2 pi |K|^2 d|K| dcos over K^2 >= 4 m^2."""
    E2 = np.sqrt(p2 * p2 + m * m)
    # K0 from its threshold 2m; |K| in [0, sqrt(K0^2 - 4m^2)]
    k0, wk0 = composite_gl((2 * m, 2 * m + 1, 2 * m + 3, 2 * m + 7, 2 * m + 15, 2 * m + 31), n_e)
    u, wu = _gl(0.0, 1.0, n_k)
    c, wc = _gl(-1.0, 1.0, n_c)
    om, wom = _gl(-7 * sigma, 7 * sigma, n_om)
    K0, U, C, OM = np.meshgrid(k0, u, c, om, indexing="ij")
    kmax = np.sqrt(np.maximum(K0 ** 2 - 4 * m * m, 0.0))
    K = U * kmax
    W = (wk0[:, None, None, None] * wu[None, :, None, None] * wc[None, None, :, None]
         * wom[None, None, None, :]) * kmax
    sK = K0 ** 2 - K ** 2
    Ein = E2 + K0 + OM
    sin_ = np.where(Ein > 0, Ein ** 2 - (p2 * p2 + K ** 2 + 2 * p2 * K * C), 0.0)
    g = np.exp(-OM ** 2 / (2 * sigma ** 2)) / (sigma * np.sqrt(TWO_PI))
    integ = np.exp(-K0 / T) * phase2(sK, m) * phase2(sin_, m) * g * TWO_PI * K ** 2
    f2 = A * np.exp(-E2 / T)
    return float(lam ** 2 * f2 * A * A / (2 * E2 * TWO_PI ** 4) * np.sum(integ * W))
