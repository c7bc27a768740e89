"""Physics pins of the oracle: one collision step from Maxwellian (or bi-Maxwellian) particles against the expected
change computed by quadrature from the method's definitions (tests/_rates.py), within three Monte-Carlo standard
errors, and the limit of that expectation as the time step goes to zero against the Landau-Fokker-Planck rates in
closed form (bi-Maxwellian isotropisation; the two-temperature exchange of Sec. 5.3, Eq. 0DSpitzer).

Setup: many cells of 8 particles per species (so that the N - 1 of intra-species pairs and the weight factors move
the rate by far more than the error bars), unit charges, eps0 = dV = 1, lnL = 10; the time step set from nu dt as the
workloads do. The standard error of the per-cell total comes from the spread of the cells around the expectation
(cells are independent). Each case states its relative standard error; a factor-of-two slip in s, a wrong reduced
mass, the wrong member of (N, N - 1), a lost weight factor or a sign error in the rotation moves a case by tens of
standard errors.

With unequal weights the scatter alone is pinned (correction off): the energy correction then moves the per-cell
rates by O(1 / N) (measured: 6% slower isotropisation and 21% faster exchange at 8 particles per species and
nu dt = 1, 3% faster exchange at 64), an effect of the method's correction rather than of the scatter; with equal
weights the correction is a no-op and the full step is pinned."""
import math

import numpy as np
import pytest
from scipy import integrate

import oracle as O

import _rates as R

LNL = 10.0
CELLS = 1 << 18


def _method(name):
    return O.N97 if name == "N97" else O.TA77


def _combos(values):
    """(probability, w_min, w_max) over independent draws of two weights, each uniform over `values`."""
    v = [float(x) for x in values]
    p = 1.0 / (len(v) ** 2)
    return [(p, min(a, b), max(a, b)) for a in v for b in v]


def _isotropisation(nu_dt, method, weights=(1.0,), correct=True, N=8, C=CELLS, seed=11, Tx=2.0, Tp=1.0):
    """One step of one species (m = 1) from the bi-Maxwellian (Tx, Tp, Tp). Returns the per-cell changes of
    sum w m v_x^2, their expectation (finite time step) and the Landau limit."""
    rng = np.random.default_rng(seed)
    m = 1.0
    v_t = math.sqrt((Tx + 2 * Tp) / 3 / m)
    dt = nu_dt / (LNL * N * np.mean(weights) / (4 * math.pi * m ** 2 * v_t ** 3))
    vx = rng.normal(0, math.sqrt(Tx / m), C * N)
    vy = rng.normal(0, math.sqrt(Tp / m), C * N)
    vz = rng.normal(0, math.sqrt(Tp / m), C * N)
    w = rng.choice(np.asarray(weights, dtype=np.float64), C * N)
    st = O.State(vx.copy(), vy.copy(), vz.copy(), w, np.arange(C + 1, dtype=np.int64) * N, C, 1)
    O.step(st, [-1.0], [m], LNL, O.Params(method=_method(method), dt=dt, seed=seed, correct=correct), n_steps=1)
    d = (m * w * (st.v()[:, 0] ** 2 - vx ** 2)).reshape(C, N).sum(1)
    k0 = LNL * dt / (4 * math.pi * (m / 2) ** 2) * (N - 1)  # s u^3 per unit w_max: intra-species N_min = N - 1
    E = N / 2 * sum(p * lo * R.iso_pair_expectation(k0 * hi, Tx, Tp, m, method) for p, lo, hi in _combos(weights))
    L = N / 2 * sum(p * lo * R.iso_pair_landau(k0 * hi, Tx, Tp, m) for p, lo, hi in _combos(weights))
    return d, E, L


def _exchange(nu_dt, method, we=(1.0,), wi=(1.0,), correct=True, N=8, C=CELLS, seed=12, M=25.0, Te=1.0, Ti=0.25):
    """One step of the electron-ion interaction alone (N electrons of mass 1 and N ions of mass M per cell, unit
    charges) from Maxwellians at Te and Ti. Returns the per-cell changes of the electrons' kinetic energy, their
    expectation and the Landau (Spitzer) limit."""
    rng = np.random.default_rng(seed)
    dt = nu_dt / (LNL * N * np.mean(we) / (4 * math.pi * Te ** 1.5))
    ve = rng.normal(0, math.sqrt(Te), (C, N, 3))
    vi = rng.normal(0, math.sqrt(Ti / M), (C, N, 3))
    w_e = rng.choice(np.asarray(we, dtype=np.float64), (C, N))
    w_i = rng.choice(np.asarray(wi, dtype=np.float64), (C, N))
    v = np.concatenate([ve, vi], axis=1).reshape(-1, 3)
    w = np.concatenate([w_e, w_i], axis=1).reshape(-1)
    off = np.zeros(2 * C + 1, np.int64)
    off[1:] = np.cumsum(np.tile([N, N], C))
    st = O.State(v[:, 0].copy(), v[:, 1].copy(), v[:, 2].copy(), w, off, C, 2)
    O.step(st, [-1.0, 1.0], [1.0, M], LNL, O.Params(method=_method(method), dt=dt, seed=seed, correct=correct),
           n_steps=1, interactions=[(0, 1)])
    v1 = st.v().reshape(C, 2 * N, 3)[:, :N]
    d = 0.5 * (w_e * ((v1 ** 2).sum(2) - (ve ** 2).sum(2))).sum(1)
    mu = M / (1.0 + M)
    k0 = LNL * dt / (4 * math.pi * mu ** 2) * N  # inter-species N_min = N
    combos = [(1.0 / (len(we) * len(wi)), min(a, b), max(a, b)) for a in we for b in wi]
    E = N * sum(p * lo * R.exchange_pair_expectation(k0 * hi, Te, 1.0, Ti, M, method) for p, lo, hi in combos)
    L = N * sum(p * lo * R.exchange_pair_landau(k0 * hi, Te, 1.0, Ti, M) for p, lo, hi in combos)
    return d, E, L


def _z(d, E):
    se = math.sqrt(((d - E) ** 2).sum()) / len(d)
    return (d.mean() - E) / se, se / abs(E)


# --- the quadrature itself, against direct integration and closed forms ---

@pytest.mark.parametrize("s", [0.01, 0.5, 3.0])
def test_angle_moments_against_direct_integration(s):
    """N97: the moments of the density exp(A x) on [-1, 1] with A from its defining equation; TA77: the Gaussian
    expectation over delta. Both by adaptive quadrature."""
    A = float(R.n97_A(np.array([s]))[0])
    assert abs(1 / math.tanh(A) - 1 / A - math.exp(-s)) < 1e-13
    Z = integrate.quad(lambda x: math.exp(A * (x - 1)), -1, 1, epsabs=0, epsrel=1e-13)[0]
    mom = lambda f: integrate.quad(lambda x: f(x) * math.exp(A * (x - 1)), -1, 1, epsabs=0, epsrel=1e-13)[0] / Z
    want = (mom(lambda x: 1 - x), mom(lambda x: (1 - x) ** 2), mom(lambda x: 1 - x * x))
    got = [float(g[0]) for g in R.angle_moments(np.array([s]), "N97")]
    np.testing.assert_allclose(got, want, rtol=1e-9)
    sd = math.sqrt(s / 2)
    g = lambda f: integrate.quad(lambda d: f(d) * math.exp(-d * d / (2 * sd * sd)) / (sd * math.sqrt(2 * math.pi)),
                                 -np.inf, np.inf, epsabs=0, epsrel=1e-12)[0]
    want = (g(lambda d: 2 * d * d / (1 + d * d)), g(lambda d: (2 * d * d / (1 + d * d)) ** 2),
            g(lambda d: (2 * d / (1 + d * d)) ** 2))
    got = [float(x[0]) for x in R.angle_moments(np.array([s]), "TA77")]
    np.testing.assert_allclose(got, want, rtol=1e-8)


def test_angle_moment_limits():
    """Small s: <1 - cos> -> s and <sin^2> -> 2 s for both samplers (s = <theta^2> / 2); large s (N97): the
    isotropic values 1, 4/3, 2/3."""
    for method in ("N97", "TA77"):
        omc, _, sin2 = R.angle_moments(np.array([1e-6]), method)
        assert abs(omc[0] / 1e-6 - 1) < 1e-5 and abs(sin2[0] / 2e-6 - 1) < 1e-5
    np.testing.assert_allclose([x[0] for x in R.angle_moments(np.array([200.0]), "N97")], [1, 4 / 3, 2 / 3],
                               rtol=1e-12)


@pytest.mark.parametrize("Tx,Tp", [(2.0, 1.0), (1.0, 3.0)])
def test_landau_closed_form(Tx, Tp):
    """The closed form of the isotropisation integral (both signs of the anisotropy) against adaptive quadrature of
    its one-dimensional form, and the finite-step quadrature's s -> 0 limit against it."""
    sx2, sp2 = 2 * Tx, 2 * Tp
    f = lambda t: (1 - 3 * t * t) / (t * t / sx2 + (1 - t * t) / sp2)
    direct = 0.5 * (2 * math.pi) ** -0.5 / (math.sqrt(sx2) * sp2) * integrate.quad(f, -1, 1, epsrel=1e-13)[0]
    assert abs(R.iso_pair_landau(1.0, Tx, Tp, 1.0) / direct - 1) < 1e-12
    for method in ("N97", "TA77"):
        k = 1e-7
        assert abs(R.iso_pair_expectation(k, Tx, Tp, 1.0, method) / R.iso_pair_landau(k, Tx, Tp, 1.0) - 1) < 1e-6
    assert R.iso_pair_landau(1.0, 1.5, 1.5, 1.0) == 0.0


def test_exchange_landau_is_spitzer():
    """The s -> 0 exchange expectation equals the Spitzer form (any mass ratio) and the finite-step quadrature tends
    to it."""
    for (Ta, ma, Tb, mb) in [(1.0, 1.0, 0.25, 25.0), (2.0, 1.0, 3.0, 1836.0), (1.0, 4.0, 1.0, 4.0)]:
        mu = ma * mb / (ma + mb)
        spitzer = (mu * math.sqrt(2 / math.pi) * ma * mb * (Tb - Ta) * math.sqrt(ma * mb)
                   / ((ma + mb) * (ma * Tb + mb * Ta) ** 1.5))
        assert abs(R.exchange_pair_landau(1.0, Ta, ma, Tb, mb) - spitzer) <= 1e-12 * abs(spitzer) + 1e-300
        if Ta != Tb:
            k = 1e-8
            assert abs(R.exchange_pair_expectation(k, Ta, ma, Tb, mb, "N97") / R.exchange_pair_landau(k, Ta, ma, Tb, mb)
                       - 1) < 1e-4


# --- the oracle against the expectations ---

@pytest.mark.parametrize("method,nu_dt", [("N97", 1.0), ("N97", 0.1), ("TA77", 1.0), ("TA77", 0.1)])
def test_isotropisation_one_step(method, nu_dt):
    d, E, _ = _isotropisation(nu_dt, method)
    z, rel = _z(d, E)
    assert rel < 0.03, rel
    assert abs(z) < 3.0, (z, d.mean(), E)


def test_isotropisation_weighted_scatter():
    """Weights 1 and 4: the lighter particle always moves, the heavier with probability w_min / w_max, s with
    w_max (correction off: the scatter alone)."""
    d, E, _ = _isotropisation(1.0, "N97", weights=(1.0, 4.0), correct=False)
    z, rel = _z(d, E)
    assert rel < 0.02 and abs(z) < 3.0, (z, rel)


def test_isotropisation_lfp_rate():
    """At nu dt = 0.02 the one-step change is within Monte-Carlo error of the Landau-Fokker-Planck isotropisation
    rate of the bi-Maxwellian itself (the finite-step expectation is 1.7% below it, under one standard error)."""
    d, E, L = _isotropisation(0.02, "N97")
    z, rel = _z(d, L)
    assert rel < 0.05 and abs(z) < 3.0, (z, rel)
    assert abs(E / L - 1) < rel


@pytest.mark.parametrize("method,nu_dt", [("N97", 1.0), ("N97", 0.1), ("TA77", 1.0)])
def test_exchange_one_step(method, nu_dt):
    d, E, _ = _exchange(nu_dt, method)
    z, rel = _z(d, E)
    assert rel < 0.03, rel
    assert abs(z) < 3.0, (z, d.mean(), E)


def test_exchange_weighted_scatter():
    d, E, _ = _exchange(1.0, "N97", we=(1.0, 4.0), wi=(1.0, 2.0), correct=False)
    z, rel = _z(d, E)
    assert rel < 0.02 and abs(z) < 3.0, (z, rel)
