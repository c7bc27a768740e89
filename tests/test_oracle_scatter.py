"""Pins for the oracle's scattering: angle samplers, rotation, and the expected-value identities of the weighted
order-N method (CPU only).

Independent references: scipy root finding / quadrature / Gauss-Hermite for the sampler moments, and brute-force
N x N expectations written from the pair kinematics (m_a dv_i = mu du, Sec. 2.1; Eqs. sb_TA_weighted and
sa_TA77_weighted) for the Monte-Carlo means.
"""
import math

import mpmath
import numpy as np
import pytest
from scipy import integrate

import oracle as O
from paper_2407_19151_gb300 import workloads as W


def L_ref(A):
    return 1.0 / math.tanh(A) - 1.0 / A


def A_ref(s):
    """Root of coth(A) - 1/A = exp(-s) in 40-digit arithmetic (mpmath), independent of the oracle's solver."""
    with mpmath.workdps(40):
        y = mpmath.exp(-mpmath.mpf(s))
        f = lambda a: mpmath.coth(a) - 1 / a - y
        lo, hi = mpmath.mpf("1e-30"), 1 / (1 - y) + 10
        return float(mpmath.findroot(f, (lo, hi), solver="anderson"))


@pytest.mark.parametrize("s", [1e-9, 1e-7, 1e-4, 1e-2, 0.1, 0.5, 1.0, 3.0, 6.0])
def test_n97_root_matches_independent_solve(s):
    # full relative precision also for tiny s (A ~ 1/s), where solving with exp(-s) would lose digits
    A = O.n97_A(s)
    assert A == pytest.approx(A_ref(s), rel=1e-13)


def test_n97_limits():
    for s in [1e-6, 1e-5]:
        assert O.n97_A(s) == pytest.approx(1.0 / s, rel=2 * s)       # A -> 1/s as s -> 0
    for s in [12.0, 20.0, 40.0]:
        assert O.n97_A(s) == pytest.approx(3.0 * math.exp(-s), rel=1e-4)  # A -> 3 exp(-s) as s -> inf
    assert O.n97_A(1e4) == 0.0                                        # exp(-s) underflows: isotropic


def test_n97_series_branch_matches_closed_form():
    # the Laurent-series branch (A < 1/2) and the closed form agree where both are accurate
    for A in np.linspace(0.3, 0.4999, 9):
        assert O.n97_L(A) == pytest.approx(L_ref(A), rel=3e-14)
    for A in [1e-3, 1e-2, 0.1]:
        assert O.n97_L(A) == pytest.approx(A / 3 - A ** 3 / 45 + 2 * A ** 5 / 945, rel=1e-6 * A)


@pytest.mark.parametrize("s", [1e-3, 0.05, 0.5, 3.0, 10.0])
def test_n97_mean_cos_is_exp_minus_s(s):
    # midpoint rule over the inverse-CDF variable: E[cos chi] = exp(-s), E[cos^2 chi] = 1 - 2 exp(-s)/A
    n = 200000
    V = (np.arange(n) + 0.5) / n
    omc = np.array([O.angle(O.N97, s, v, 0.5)[1] for v in V[:: n // 4000]])
    V2 = V[:: n // 4000]
    # coarse grid for speed; refine with quad for the exact check
    A = A_ref(s)
    f = lambda v: -math.log1p(v * math.expm1(-2 * A)) / A
    m1 = integrate.quad(lambda v: 1 - f(v), 0, 1, limit=200)[0]
    assert m1 == pytest.approx(math.exp(-s), rel=1e-8, abs=1e-12)
    assert np.mean(1 - omc) == pytest.approx(math.exp(-s), abs=2e-3)
    # the oracle's sampler equals the inverse CDF evaluated with the independently solved A
    for v in [0.01, 0.3, 0.77, 0.999]:
        assert O.angle(O.N97, s, v, 0.5)[1] == pytest.approx(f(v), rel=1e-10, abs=1e-15)
    st, omc1 = O.angle(O.N97, s, 0.3, 0.5)
    assert st ** 2 == pytest.approx(omc1 * (2 - omc1), rel=1e-12)
    # sin chi near back-scatter equals the 40-digit value of sqrt((1 - cos)(1 + cos)) from the inverse CDF
    with mpmath.workdps(40):
        Am = mpmath.mpf(A)
        for v in [0.999, 0.9999999]:
            cosx = 1 + mpmath.log(mpmath.mpf(1 - v) + mpmath.mpf(v) * mpmath.exp(-2 * Am)) / Am
            ref = float(mpmath.sqrt((1 - cosx) * (1 + cosx)))
            assert O.angle(O.N97, s, v, 0.5)[0] == pytest.approx(ref, rel=1e-9, abs=1e-300)


@pytest.mark.parametrize("s", [1e-3, 0.05, 0.3])
def test_n97_cos_accurate_when_A_times_angle_is_large(s):
    """Large A with V near 1 puts 1 + V expm1(-2A) close to zero; 1 - cos chi must still be accurate (40-digit
    reference of -ln(1 - V + V exp(-2A)) / A)."""
    A = O.n97_A(s)
    with mpmath.workdps(40):
        Am = mpmath.mpf(A)
        for v in [0.9, 0.999, 1 - 2.0 ** -23]:
            ref = float(-mpmath.log(1 - mpmath.mpf(v) + mpmath.mpf(v) * mpmath.exp(-2 * Am)) / Am)
            assert O.angle(O.N97, s, v, 0.5)[1] == pytest.approx(ref, rel=1e-12)


@pytest.mark.parametrize("s", [1e-3, 0.05, 0.8])
def test_ta77_delta_variance(s):
    rng = np.random.default_rng(1)
    U1 = (np.floor(rng.random(40000) * 2**23) + 0.5) / 2**23
    U4 = (np.floor(rng.random(40000) * 2**23) + 0.5) / 2**23
    d = []
    for a, b in zip(U1, U4):
        st, omc = O.angle(O.TA77, s, a, b)
        d.append(st / (2.0 - omc))  # tan(Theta/2) = sin / (1 + cos)
    d = np.array(d)
    assert np.mean(d ** 2) == pytest.approx(s / 2, rel=0.03)          # <delta^2> = s/2
    assert abs(np.mean(d)) < 4 * math.sqrt(s / 2 / len(d))              # symmetric
    # each sample equals sqrt(s/2) * Box-Muller(U1, U4)
    g = np.sqrt(-2 * np.log(U1[:50])) * np.cos(2 * np.pi * U4[:50])
    np.testing.assert_allclose(d[:50], np.sqrt(s / 2) * g, rtol=1e-12, atol=1e-300)


def test_rotation_invariants():
    rng = np.random.default_rng(2)
    for _ in range(200):
        u = rng.normal(size=3)
        theta = rng.uniform(0, math.pi)
        phi = rng.uniform(0, 2 * math.pi)
        du = O.rotate(u, math.sin(theta), 1 - math.cos(theta), phi)
        up = u + du
        assert np.linalg.norm(up) == pytest.approx(np.linalg.norm(u), rel=1e-13)
        assert np.dot(u, up) / np.dot(u, u) == pytest.approx(math.cos(theta), abs=1e-13)
    # azimuth: phi and phi + pi/2 give orthogonal perpendicular parts
    u = np.array([0.3, -0.7, 0.5])
    a = O.rotate(u, 0.6, 1 - 0.8, 0.4) + u
    b = O.rotate(u, 0.6, 1 - 0.8, 0.4 + math.pi / 2) + u
    uh = u / np.linalg.norm(u)
    pa, pb = a - np.dot(a, uh) * uh, b - np.dot(b, uh) * uh
    assert abs(np.dot(pa, pb)) < 1e-13
    # u along z: the degenerate branch still preserves |u| and the angle
    for uz in [2.0, -2.0]:
        u = np.array([0.0, 0.0, uz])
        up = u + O.rotate(u, 0.6, 0.2, 1.1)
        assert np.linalg.norm(up) == pytest.approx(2.0, rel=1e-14)
        assert np.dot(u, up) / 4.0 == pytest.approx(0.8, abs=1e-14)


# ------------------------------------------------------------------------------ expected values of the scatter
def h1_exact(method, s):
    """E[1 - cos Theta] for a pair with scattering length s."""
    if method == O.N97:
        return -math.expm1(-s)
    x, wts = np.polynomial.hermite.hermgauss(80)
    d = np.sqrt(s) * x  # delta ~ N(0, s/2)
    return float(np.sum(wts * 2 * d ** 2 / (1 + d ** 2)) / math.sqrt(math.pi))


def sin2_exact(method, s):
    """E[sin^2 Theta]."""
    if method == O.N97:
        return 2.0 * math.exp(-s) / A_ref(s)
    x, wts = np.polynomial.hermite.hermgauss(80)
    d = np.sqrt(s) * x
    return float(np.sum(wts * (2 * d / (1 + d ** 2)) ** 2) / math.sqrt(math.pi))


def replicate(v, w, counts, M):
    """M copies of one cell (different cell ids -> independent draws)."""
    counts = np.asarray(counts)
    S = len(counts)
    off = np.concatenate([[0], np.cumsum(np.tile(counts, M))]).astype(np.int64)
    V = np.tile(v, (M, 1))
    return O.State(V[:, 0], V[:, 1], V[:, 2], np.tile(w, M), off, M, S)


@pytest.mark.parametrize("method", [O.TA77, O.N97])
def test_weighted_drag_expectation(method):
    """Mean dv of every particle over many draws equals the exact expectation of the weighted order-N rule:
    partner uniform (N_a = N_b), lighter particle always moves, heavier one with probability w_min/w_max
    [Eqs. sb_TA_weighted, sa_TA77_weighted]; at small s this is the N x N / LFP drag of Eq. LDF_drag."""
    rng = np.random.default_rng(7)
    n = 4
    ma, mb, qa, qb = 1.0, 4.0, -1.0, 2.0
    v = rng.normal(size=(2 * n, 3))
    v[n:] *= 0.5
    w = np.array([1.0, 3.0, 10.0, 0.5, 2.0, 2.0, 7.0, 0.3])
    M = 30000
    st = replicate(v, w, [n, n], M)
    lnL = 10.0
    dt = 2e-3
    p = O.Params(method=method, dt=dt, correct=False, seed=99)
    O.scatter(st, [qa, qb], [ma, mb], lnL, 0, 1, 0, p)
    dv = (st.v() - np.tile(v, (M, 1))).reshape(M, 2 * n, 3)
    mean, se = dv.mean(axis=0), dv.std(axis=0) / math.sqrt(M)
    mu = ma * mb / (ma + mb)

    def expectations(dt_):
        kappa = qa ** 2 * qb ** 2 * lnL * dt_ / (4 * math.pi)
        exact = np.zeros((2 * n, 3))
        lfp = np.zeros((2 * n, 3))
        for i in range(n):
            for j in range(n, 2 * n):
                u = v[i] - v[j]
                um = np.linalg.norm(u)
                wmax, wmin = max(w[i], w[j]), min(w[i], w[j])
                s = kappa / mu ** 2 * wmax * n / um ** 3
                Pi = 1.0 if w[i] <= w[j] else wmin / wmax
                Pj = 1.0 if w[j] <= w[i] else wmin / wmax
                h = h1_exact(method, s)
                exact[i] += (1 / n) * Pi * (mu / ma) * (-u) * h
                exact[j] += (1 / n) * Pj * (mu / mb) * (u) * h
                # Eq. sij_sji: s_ij uses w_j, s_ji uses w_i; Eq. LDF_drag sums u s over all partners
                lfp[i] += -(mu / ma) * u * (kappa / mu ** 2 * w[j] / um ** 3)
                lfp[j] += (mu / mb) * u * (kappa / mu ** 2 * w[i] / um ** 3)
        return exact, lfp

    exp_exact, _ = expectations(dt)
    z = (mean - exp_exact) / se
    assert np.all(np.abs(z) < 5.0), z
    # small-s limit: the exact expectation of the weighted order-N rule is the LFP drag
    ex_small, lfp_small = expectations(1e-10)
    rel = np.linalg.norm(ex_small - lfp_small, axis=1) / np.linalg.norm(lfp_small, axis=1)
    assert rel.max() < 1e-4


@pytest.mark.parametrize("method", [O.TA77, O.N97])
def test_isotropisation_expectation(method):
    """Equal weights, one species, even N: E[d sum m w v_x^2] = sum_{i<j} m w sin^2-moment (u^2 - 3 u_x^2)/4/(N-1)."""
    rng = np.random.default_rng(11)
    n = 8
    v = rng.normal(size=(n, 3)) * np.array([math.sqrt(2.0), 1.0, 1.0])
    w = np.full(n, 2.0)
    M = 20000
    st = replicate(v, w, [n], M)
    lnL, dt = 10.0, 4e-3
    p = O.Params(method=method, dt=dt, correct=False, seed=5)
    O.scatter(st, [-1.0], [1.0], lnL, 0, 0, 0, p)
    vx_after = st.vx.reshape(M, n)
    d = (2.0 * (vx_after ** 2 - v[:, 0] ** 2)).sum(axis=1)
    kappa = lnL * dt / (4 * math.pi)
    mu = 0.5
    expect = 0.0
    for i in range(n):
        for j in range(i + 1, n):
            u = v[i] - v[j]
            um = np.linalg.norm(u)
            s = kappa / mu ** 2 * 2.0 * (n - 1) / um ** 3
            expect += 2.0 * 0.25 * sin2_exact(method, s) * (um ** 2 - 3 * u[0] ** 2) / (n - 1)
    z = (d.mean() - expect) / (d.std() / math.sqrt(M))
    assert abs(z) < 5.0, (d.mean(), expect)
    assert expect < 0  # the hot x direction cools


@pytest.mark.parametrize("method", [O.TA77, O.N97])
def test_equilibration_expectation(method):
    """Two species, N_a = N_b, unequal weights: E[dKE_a] = sum_ij (1/N) P_i w_i mu h (-v_i.u + (mu/m_a) u^2)."""
    rng = np.random.default_rng(13)
    n = 4
    ma, mb = 1.0, 10.0
    v = np.vstack([rng.normal(size=(n, 3)) * 1.0, rng.normal(size=(n, 3)) * math.sqrt(4.0 / mb)])
    w = np.array([1.0, 1.0, 1.0, 1.0, 3.0, 20.0, 50.0, 8.0])
    M = 30000
    st = replicate(v, w, [n, n], M)
    lnL, dt = 10.0, 2e-3
    p = O.Params(method=method, dt=dt, correct=False, seed=21)
    O.scatter(st, [-1.0, 1.0], [ma, mb], lnL, 0, 1, 0, p)
    va = st.v().reshape(M, 2 * n, 3)[:, :n]
    dKE = (0.5 * ma * w[:n, None] * (va ** 2 - v[:n] ** 2)).sum(axis=(1, 2))
    mu = ma * mb / (ma + mb)
    kappa = lnL * dt / (4 * math.pi)
    expect = 0.0
    for i in range(n):
        for j in range(n, 2 * n):
            u = v[i] - v[j]
            um = np.linalg.norm(u)
            s = kappa / mu ** 2 * max(w[i], w[j]) * n / um ** 3
            Pi = 1.0 if w[i] <= w[j] else w[j] / w[i]
            expect += (1 / n) * Pi * w[i] * mu * h1_exact(method, s) * (-np.dot(v[i], u) + mu / ma * um ** 2)
    z = (dKE.mean() - expect) / (dKE.std() / math.sqrt(M))
    assert abs(z) < 5.0, (dKE.mean(), expect)


def test_relativistic_pair_conserves_four_momentum():
    rng = np.random.default_rng(3)
    c = 1.0
    for _ in range(100):
        ma, mb = 1.0, rng.choice([1.0, 1836.0])
        ui = rng.normal(size=3) * rng.choice([0.01, 1.0, 5.0])
        uj = rng.normal(size=3) * 0.1
        th, ph = rng.uniform(0, math.pi), rng.uniform(0, 2 * math.pi)
        dp, pstar, vrel = O.rel_scatter_dp(c, ma, mb, ui, uj, math.sin(th), 1 - math.cos(th), ph)
        ui2, uj2 = ui + dp / ma, uj - dp / mb
        E = lambda m, u: m * math.sqrt(1 + np.dot(u, u) / c ** 2)
        Ebefore = E(ma, ui) + E(mb, uj)
        assert E(ma, ui2) + E(mb, uj2) == pytest.approx(Ebefore, rel=1e-12)
        assert vrel > 0 and pstar > 0


def test_relativistic_scatter_reduces_to_classical():
    # c -> infinity: dp -> mu du of the non-relativistic rotation; |p*| -> mu u; v_rel* -> u
    ma, mb = 1.0, 3.0
    vi, vj = np.array([0.3, -0.2, 0.5]), np.array([-0.1, 0.4, 0.05])
    mu = ma * mb / (ma + mb)
    u = vi - vj
    du = O.rotate(u, 0.3, 1 - math.sqrt(1 - 0.09), 0.7)
    dp, pstar, vrel = O.rel_scatter_dp(1e6, ma, mb, vi, vj, 0.3, 1 - math.sqrt(1 - 0.09), 0.7)
    np.testing.assert_allclose(dp, mu * du, rtol=1e-9, atol=1e-15)
    assert pstar == pytest.approx(mu * np.linalg.norm(u), rel=1e-10)
    assert vrel == pytest.approx(np.linalg.norm(u), rel=1e-10)


def test_duplicity_weighting_pins():
    """Duplicity weighting (the alternative of Higginson et al. described in Sec. 3.2): s uses (w_max / D_ij) N_max for
    inter-species pairs, D_ij = how often the smaller population's particle of the pair is paired. One cell with
    N_a = 3, N_b = 2 and unit weights: pairs 0 and 2 share b's first particle (D = 2), pair 1 has D = 1, so s is the
    paper's s times 3/4 and 3/2. The scatter with duplicity weighting therefore equals, particle by particle, the
    paper's scatter with lnL scaled by 3/4 (particles of pairs 0 and 2) and by 3/2 (particles of pair 1)."""
    rng = np.random.default_rng(8)
    counts = np.array([[3, 2]])
    off = np.array([0, 3, 5], dtype=np.int64)
    v = rng.standard_normal((5, 3))
    w = np.ones(5)
    q, m = np.array([-1.0, 1.0]), np.array([1.0, 4.0])

    def run(weighting, lnl):
        st = O.State(v[:, 0], v[:, 1], v[:, 2], w, off, 1, 2)
        p = O.Params(method=O.TA77, dt=0.3, seed=21, step=2, correct=False, weighting=weighting)
        O.step(st, q, m, np.full((2, 2), lnl), p, interactions=[(0, 1)])
        return st.v()

    pi, pj, fl = O.pairs(off, 1, 2, 0, 1, 0, 21, 2)
    shared = {int(pi[0]), int(pj[0]), int(pi[2]), int(pj[2])}
    single = {int(pi[1]), int(pj[1])}
    assert int(pj[0]) == int(pj[2]) and not (shared & single)
    h = run(1, 10.0)
    for idx, scale in ((sorted(shared), 0.75), (sorted(single), 1.5)):
        ref = run(0, 10.0 * scale)
        np.testing.assert_allclose(h[idx], ref[idx], rtol=0, atol=1e-12 * np.abs(v).max())
    # equal to the paper's s when N_min divides N_max in every cell (then D_ij = N_max / N_min for every pair)
    wl = W.differentiable(n_cells=6, per_species=8)
    wl.counts[:, 0] = 16
    wl2 = W.differentiable(n_cells=6, per_species=16)
    vx = np.concatenate([wl2.vx.reshape(6, 32)[:, :16], wl.vx.reshape(6, 16)[:, 8:]], axis=1).ravel()
    vy = np.concatenate([wl2.vy.reshape(6, 32)[:, :16], wl.vy.reshape(6, 16)[:, 8:]], axis=1).ravel()
    vz = np.concatenate([wl2.vz.reshape(6, 32)[:, :16], wl.vz.reshape(6, 16)[:, 8:]], axis=1).ravel()
    ww = np.concatenate([wl2.w.reshape(6, 32)[:, :16], wl.w.reshape(6, 16)[:, 8:]], axis=1).ravel()
    off2 = np.zeros(13, dtype=np.int64)
    off2[1:] = np.cumsum(np.tile([16, 8], 6))
    out = []
    for weighting in (0, 1):
        st = O.State(vx, vy, vz, ww, off2, 6, 2)
        O.step(st, wl.q, wl.m, wl.lnL, O.Params(method=O.N97, dt=wl.dt * 20, seed=3, weighting=weighting))
        out.append(st.v())
    np.testing.assert_allclose(out[1], out[0], rtol=0, atol=1e-12 * np.abs(out[0]).max())


@pytest.mark.parametrize("na,nb,intra", [(2, 0, True), (3, 0, True), (8, 0, True), (9, 0, True), (1, 1, False),
                                         (3, 5, False), (5, 3, False), (4, 4, False), (7, 2, False)])
def test_nxn_schedule_covers_every_pair_once(na, nb, intra):
    """Order N x N pairing (Sec. 3.1): every pair of the cell exactly once per step, the pairs of a round disjoint."""
    sched = O.nxn_schedule(na, nb, intra)
    pairs = [(min(a, b), max(a, b)) if intra else (a, b) for _, _, a, b in sched]
    want = ({(i, j) for i in range(na) for j in range(i + 1, na)} if intra else
            {(i, j) for i in range(na) for j in range(nb)})
    assert len(pairs) == len(want) and set(pairs) == want
    rounds = {}
    for _, r, a, b in sched:
        rounds.setdefault(r, []).append((("a", a), ("a" if intra else "b", b)))
    for r, ps in rounds.items():
        touched = [x for p in ps for x in p]
        assert len(touched) == len(set(touched)), r


@pytest.mark.parametrize("method", [O.TA77, O.N97])
def test_nxn_drag_expectation(method):
    """Mean dv of every particle over many draws in the order N x N mode equals the sum over all partners of the
    single-pair expectation with s = kappa w_max / (mu^2 u^3) (Eq. sab_weighted) and the rejection of the heavier
    particle. Species b drifts by 3 so that every pair has s < 1e-2: the order of a particle's pairs within the step
    is then a second-order effect."""
    rng = np.random.default_rng(7)
    n = 4
    ma, mb, qa, qb = 1.0, 4.0, -1.0, 2.0
    v = rng.normal(size=(2 * n, 3))
    v[n:] *= 0.5
    v[n:, 0] += 3.0
    w = np.array([1.0, 3.0, 10.0, 0.5, 2.0, 2.0, 7.0, 0.3])
    M = 30000
    st = replicate(v, w, [n, n], M)
    lnL, dt = 10.0, 2e-3
    p = O.Params(method=method, dt=dt, correct=False, seed=99, pairing=1)
    O.scatter(st, [qa, qb], [ma, mb], lnL, 0, 1, 0, p)
    dv = (st.v() - np.tile(v, (M, 1))).reshape(M, 2 * n, 3)
    mean, se = dv.mean(axis=0), dv.std(axis=0) / math.sqrt(M)
    mu = ma * mb / (ma + mb)
    kappa = qa ** 2 * qb ** 2 * lnL * dt / (4 * math.pi)
    exact = np.zeros((2 * n, 3))
    for i in range(n):
        for j in range(n, 2 * n):
            u = v[i] - v[j]
            um = np.linalg.norm(u)
            wmax, wmin = max(w[i], w[j]), min(w[i], w[j])
            s = kappa / mu ** 2 * wmax / um ** 3
            Pi = 1.0 if w[i] <= w[j] else wmin / wmax
            Pj = 1.0 if w[j] <= w[i] else wmin / wmax
            assert s < 1e-2
            h = h1_exact(method, s)
            exact[i] += Pi * (mu / ma) * (-u) * h
            exact[j] += Pj * (mu / mb) * (u) * h
    z = (mean - exact) / se
    assert np.all(np.abs(z) < 5.0), z


def test_nxn_equal_weights_conserve_pairwise():
    """Equal weights: every N x N pair conserves momentum and energy, so the scatter alone conserves them per cell."""
    wl = W.differentiable(n_cells=4, per_species=10)
    wl.w[:] = 3.0
    st = O.State(wl.vx, wl.vy, wl.vz, wl.w, wl.offsets, wl.n_cells, wl.n_species)
    v0 = st.v().copy()
    O.step(st, wl.q, wl.m, wl.lnL, O.Params(method=O.N97, dt=wl.dt * 50, seed=4, correct=False, pairing=1))
    v1 = st.v()
    sp = wl.species_of_particles()
    mw = wl.m[sp] * wl.w
    cells = np.repeat(np.arange(wl.n_cells), np.diff(wl.offsets[::wl.n_species]))
    for c in range(wl.n_cells):
        k = cells == c
        P0, P1 = (mw[k, None] * v0[k]).sum(0), (mw[k, None] * v1[k]).sum(0)
        E0, E1 = (mw[k] * (v0[k] ** 2).sum(1)).sum(), (mw[k] * (v1[k] ** 2).sum(1)).sum()
        assert np.abs(P1 - P0).max() < 1e-12 * np.abs(mw[k, None] * v0[k]).sum()
        assert abs(E1 - E0) < 1e-12 * E0
    assert np.abs(v1 - v0).max() > 1e-3


def _boost_to_cm(mp, c, ma, mb, ui, uj):
    """Lorentz boost (50-digit mpmath) into the pair's centre-of-momentum frame, built from 4-momenta: returns a
    function mapping a lab 3-momentum of mass m to its CM 3-momentum."""
    c = mp.mpf(c)
    pa = [mp.mpf(ma) * mp.mpf(x) for x in ui]
    pb = [mp.mpf(mb) * mp.mpf(x) for x in uj]
    Ea = mp.sqrt((mp.mpf(ma) * c ** 2) ** 2 + sum(x * x for x in pa) * c ** 2)
    Eb = mp.sqrt((mp.mpf(mb) * c ** 2) ** 2 + sum(x * x for x in pb) * c ** 2)
    P = [x + y for x, y in zip(pa, pb)]
    beta = [x * c / (Ea + Eb) for x in P]
    b2 = sum(x * x for x in beta)
    g = 1 / mp.sqrt(1 - b2)

    def to_cm(p, m):
        E = mp.sqrt((mp.mpf(m) * c ** 2) ** 2 + sum(x * x for x in p) * c ** 2)
        bp = sum(b * x for b, x in zip(beta, p))
        # p' = p + ((g - 1) (beta.p) / b^2 - g E / c) beta
        k = (g - 1) * bp / b2 - g * E / c if b2 > 0 else 0
        return [x + k * b for x, b in zip(p, beta)], E

    return to_cm, pa, pb


def test_relativistic_scatter_is_an_elastic_cm_rotation_by_theta():
    """The relativistic scatter (a reading: the paper prints no kinematics) checked against its definition by an
    independent route: 50-digit Lorentz boosts of the oracle's pre- and post-collision momenta into the pair's CM
    frame. There the momenta stay opposite and keep their magnitude |p*| (elastic), turn by exactly Theta, the
    azimuths phi and phi + pi mirror each other about p*, and v_rel* is the difference of the two CM velocities."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 50
    rng = np.random.default_rng(17)
    c = 1.0
    for trial in range(40):
        ma, mb = 1.0, float(rng.choice([1.0, 1836.0, 7.5]))
        ui = rng.normal(size=3) * rng.choice([0.01, 1.0, 5.0])
        uj = rng.normal(size=3) * rng.choice([0.1, 3.0])
        th = rng.uniform(0.01, math.pi - 0.01)
        ph = rng.uniform(0, 2 * math.pi)
        st, omc = math.sin(th), 1 - math.cos(th)
        to_cm, pa, pb = _boost_to_cm(mp, c, ma, mb, ui, uj)
        sa, _ = to_cm(pa, ma)
        sb, _ = to_cm(pb, mb)
        assert max(abs(x + y) for x, y in zip(sa, sb)) < mp.mpf(1e-40) * (1 + mp.norm(sa))  # opposite in the CM
        pstar = mp.norm(sa)
        outs = []
        for phi in (ph, ph + math.pi):
            dp, pm, vrel = O.rel_scatter_dp(c, ma, mb, ui, uj, st, omc, phi)
            pa2 = [x + mp.mpf(d) for x, d in zip(pa, dp)]
            pb2 = [x - mp.mpf(d) for x, d in zip(pb, dp)]
            sa2, _ = to_cm(pa2, ma)
            sb2, _ = to_cm(pb2, mb)
            tol = 1e-12 * float(pstar) + 1e-13 * float(mp.norm(pa) + mp.norm(pb))
            assert float(mp.norm([x + y for x, y in zip(sa2, sb2)])) < tol
            assert abs(float(mp.norm(sa2) - pstar)) < tol
            cos_turn = sum(x * y for x, y in zip(sa, sa2)) / (pstar * mp.norm(sa2))
            assert abs(float(cos_turn) - math.cos(th)) < 1e-10 * (1 + float(mp.norm(pa) + mp.norm(pb)) / float(pstar))
            assert pm == pytest.approx(float(pstar), rel=1e-12)
            # v_rel* = |v_a* - v_b*| with v* = p* c^2 / E*
            Ea_cm = mp.sqrt((mp.mpf(ma) * c ** 2) ** 2 + pstar ** 2 * c ** 2)
            Eb_cm = mp.sqrt((mp.mpf(mb) * c ** 2) ** 2 + mp.norm(sb) ** 2 * c ** 2)
            va = [x * c ** 2 / Ea_cm for x in sa]
            vb = [x * c ** 2 / Eb_cm for x in sb]
            assert vrel == pytest.approx(float(mp.norm([x - y for x, y in zip(va, vb)])), rel=1e-12)
            outs.append(sa2)
        # phi and phi + pi: the scattered momenta mirror about p*, their sum is 2 cos(Theta) p*
        mirror = [x + y - 2 * mp.cos(mp.mpf(th)) * z for x, y, z in zip(outs[0], outs[1], sa)]
        assert float(mp.norm(mirror)) < 1e-10 * (float(pstar) + float(mp.norm(pa) + mp.norm(pb)))
