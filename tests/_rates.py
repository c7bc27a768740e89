"""Expected one-step changes of the binary collision model over Maxwellian and bi-Maxwellian particle pairs, by
quadrature, for the oracle's rate pins. Written from the method's definitions, independently of the oracle:

* a pair (v_a, v_b) with relative velocity u is scattered by rotating u through the polar angle chi about a uniform
  azimuth, so that v_a += (mu / m_a) du, v_b -= (mu / m_b) du with du = u' - u (Sec. 3, Eq. sab_TA77 for s);
* with weights, the lighter-weight particle always moves and the heavier one with probability w_min / w_max, so each
  side's expected change carries the factor w_min, while s uses w_max (Sec. 3);
* TA77: delta = tan(chi / 2) is normal with variance s / 2; N97: the density of cos chi is proportional to
  exp(A cos chi) with coth A - 1 / A = exp(-s) (both follow from s = <theta^2> / 2).

Averaging the rotation over the azimuth gives, for a fixed u and s,
    E[du] = -u <1 - cos chi>,   E[du_x^2] = <(1 - cos chi)^2> u_x^2 + <sin^2 chi> (u^2 - u_x^2) / 2,
    E|du|^2 = 2 u^2 <1 - cos chi>.
As s -> 0, <1 - cos chi> -> s and <sin^2 chi> -> 2 s: the expectations become those of the Landau-Fokker-Planck
operator, which the *_landau functions give in closed form (derived here, see each docstring)."""
from __future__ import annotations

import math

import numpy as np
from scipy import special


def n97_A(s):
    """Root A of coth A - 1/A = exp(-s), vectorised (bisection in log A; the series A/3 - A^3/45 below 1e-3)."""
    s = np.asarray(s, dtype=np.float64)
    target = np.exp(-s)
    lo = np.full(s.shape, -750.0)
    hi = np.full(s.shape, 60.0)
    for _ in range(110):
        mid = 0.5 * (lo + hi)
        A = np.exp(mid)
        with np.errstate(over="ignore", divide="ignore", invalid="ignore"):
            L = np.where(A < 1e-3, A / 3 - A ** 3 / 45, 1 / np.tanh(A) - 1 / A)
        up = L < target
        lo = np.where(up, mid, lo)
        hi = np.where(up, hi, mid)
    return np.exp(0.5 * (lo + hi))


def angle_moments(s, method: str):
    """(<1 - cos chi>, <(1 - cos chi)^2>, <sin^2 chi>) of the TA77 or N97 angle for scattering parameter s.
    N97: <cos chi> = exp(-s) by construction and <cos^2 chi> = 1 - 2 <cos chi> / A (second derivative of the
    normalisation 2 sinh A / A). TA77: closed forms of the Gaussian expectations over delta."""
    s = np.asarray(s, dtype=np.float64)
    if method == "N97":
        e = np.exp(-s)
        big = s > 600.0
        A = n97_A(np.minimum(s, 600.0))
        sin2 = np.where(big, 2.0 / 3.0, 2.0 * e / np.where(big, 1.0, A))
        omc = 1.0 - e
        return omc, 2.0 * omc - sin2, sin2
    if method != "TA77":
        raise ValueError(method)
    # delta ~ N(0, s / 2), q = 1 + delta^2: 1 - cos = 2 - 2 / q, sin^2 = 4 / q - 4 / q^2, and with a = 1 / s the
    # Gaussian integrals E[1 / q] = sqrt(pi a) erfcx(sqrt(a)), E[1 / q^2] = sqrt(pi a) (1/2 - a) erfcx(sqrt(a)) + a
    # (the second from differentiating int exp(-a x^2) / (b + x^2) dx = pi b^{-1/2} exp(a b) erfc(sqrt(a b)) in b);
    # below s = 1e-3 the asymptotic series of erfcx instead (the closed forms cancel there)
    a = 1.0 / np.maximum(s, 1e-3)
    e1 = np.sqrt(np.pi * a) * special.erfcx(np.sqrt(a))
    e2 = e1 * (0.5 - a) + a
    small = s < 1e-3
    omc = np.where(small, s * (1 - s * (1.5 - s * (3.75 - s * 13.125))), 2.0 - 2.0 * e1)
    sin2 = np.where(small, s * (2 - s * (6 - s * (22.5 - s * 105.0))), 4.0 * e1 - 4.0 * e2)
    return omc, 2.0 * omc - sin2, sin2  # (1 - cos)^2 + sin^2 = 2 (1 - cos)


def _radial_nodes():
    """Nodes and weights in x = u sqrt(a) on (0, sqrt(40)): Gauss-Legendre on log-spaced panels (the integrands
    vary fastest where s ~ 1, at small u)."""
    edges = np.concatenate([[0.0], np.geomspace(1e-4, math.sqrt(40.0), 80)])
    g, gw = np.polynomial.legendre.leggauss(12)
    lo, hi = edges[:-1, None], edges[1:, None]
    return (0.5 * (hi - lo) * g + 0.5 * (hi + lo)).ravel(), (0.5 * (hi - lo) * gw).ravel()


def iso_pair_expectation(kappa: float, Tx: float, Tp: float, m: float, method: str) -> float:
    """Expected change of m (v_ax^2 + v_bx^2) for one scattered pair of equal mass m (both sides moved) drawn from the
    bi-Maxwellian with temperatures Tx (along x) and Tp (along y and z), s = kappa / u^3. The relative velocity is
    Gaussian with variances 2 Tx / m and 2 Tp / m; the change is m (u_x du_x + du_x^2 / 2). Polar coordinates about
    x (t = cos of the polar angle) with the azimuth integrated out."""
    sx2, sp2 = 2.0 * Tx / m, 2.0 * Tp / m
    x, xw = _radial_nodes()
    t, tw = np.polynomial.legendre.leggauss(64)
    t, tw = 0.5 * t + 0.5, 0.5 * tw  # t in (0, 1); the integrand is even in t
    a = t * t / (2 * sx2) + (1 - t * t) / (2 * sp2)
    u = x[None, :] / np.sqrt(a)[:, None]
    s = kappa / u ** 3
    omc, omc2, sin2 = angle_moments(s, method)
    ux2 = (u * t[:, None]) ** 2
    H = m * (-ux2 * omc + 0.5 * omc2 * ux2 + 0.25 * sin2 * (u * u - ux2))
    dens = np.exp(-x[None, :] ** 2) * u * u / np.sqrt(a)[:, None]  # e^{-a u^2} u^2 du, du = dx / sqrt(a)
    norm = 2.0 * (2 * math.pi) ** -1.5 / (math.sqrt(sx2) * sp2) * 2 * math.pi
    return float(norm * (tw[:, None] * xw[None, :] * H * dens).sum())


def iso_pair_landau(kappa: float, Tx: float, Tp: float, m: float) -> float:
    """The s -> 0 limit of iso_pair_expectation: m (kappa / 2) E[(u^2 - 3 u_x^2) / u^3]. With the u integral done,
    E = (2 pi)^{-1/2} / (sigma_x sigma_p^2) * J, J = int_{-1}^{1} (1 - 3 t^2) / (alpha + beta t^2) dt, alpha = 1 /
    sigma_p^2, beta = 1 / sigma_x^2 - alpha; and J = -6 / beta + (1 + 3 alpha / beta) * 2 I, I the integral of
    1 / (alpha + beta t^2) over (0, 1): atan(sqrt(beta / alpha)) / sqrt(alpha beta) for beta > 0, the atanh form for
    beta < 0."""
    sx2, sp2 = 2.0 * Tx / m, 2.0 * Tp / m
    alpha, beta = 1.0 / sp2, 1.0 / sx2 - 1.0 / sp2
    if abs(beta) < 1e-12 * alpha:
        return 0.0
    if beta > 0:
        I = math.atan(math.sqrt(beta / alpha)) / math.sqrt(alpha * beta)
    else:
        I = math.atanh(math.sqrt(-beta / alpha)) / math.sqrt(-alpha * beta)
    J = -6.0 / beta + (1.0 + 3.0 * alpha / beta) * 2.0 * I
    return m * 0.5 * kappa * (2 * math.pi) ** -0.5 / (math.sqrt(sx2) * sp2) * J


def exchange_pair_expectation(kappa: float, Ta: float, ma: float, Tb: float, mb: float, method: str) -> float:
    """Expected change of the kinetic energy of side a, m_a |v_a|^2 / 2, for one scattered pair of Maxwellians
    (temperatures Ta, Tb, masses ma, mb), both sides moved, s = kappa / u^3. Given u, E[dKE_a] = mu <1 - cos chi>
    (-v_a . u + (mu / m_a) u^2), and E[v_a | u] = (sa2 / (sa2 + sb2)) u for v_a, v_b Gaussian with variances sa2 =
    Ta / ma, sb2 = Tb / mb: a one-dimensional integral over the Maxwell distribution of |u|."""
    sa2, sb2 = Ta / ma, Tb / mb
    sig2 = sa2 + sb2
    mu = ma * mb / (ma + mb)
    x, xw = _radial_nodes()
    u = x * math.sqrt(2.0 * sig2)  # exp(-u^2 / (2 sig2)) = exp(-x^2)
    omc, _, _ = angle_moments(kappa / u ** 3, method)
    g = mu * omc * u * u * (mu / ma - sa2 / sig2)
    dens = math.sqrt(2.0 / math.pi) / sig2 ** 1.5 * u * u * np.exp(-x * x) * math.sqrt(2.0 * sig2)
    return float((xw * g * dens).sum())


def exchange_pair_landau(kappa: float, Ta: float, ma: float, Tb: float, mb: float) -> float:
    """The s -> 0 limit: mu kappa (mu / m_a - sa2 / sig2) E[1 / |u|], E[1 / |u|] = sqrt(2 / (pi sig2)). It equals
    mu kappa sqrt(2 / pi) ma mb (Tb - Ta) sqrt(ma mb) / ((ma + mb) (ma Tb + mb Ta)^{3/2}), the Spitzer form."""
    sa2, sb2 = Ta / ma, Tb / mb
    sig2 = sa2 + sb2
    mu = ma * mb / (ma + mb)
    return mu * kappa * (mu / ma - sa2 / sig2) * math.sqrt(2.0 / (math.pi * sig2))
