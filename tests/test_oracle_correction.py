"""Pins for the oracle's moment correction (CPU only).

Invariants fixed by the paper: the momentum shift of Eq. vp_pm restores total momentum exactly and is
proportional to each particle's weight; each zero-angle inelastic pair conserves momentum and changes the pair's
centre-of-mass energy by exactly -U (Eqs. vp1_inelastic, vp2_inelastic, consE_inelastic, vrel_inelastic; Appendix
A for relativistic particles, Eq. alpha_Eq0); the inter-species split follows Eq. DeltaEs; equal weights need no
correction (Sec. 3.1); the first-order form of Eqs. vp1_inelastic_2 / vp2_inelastic_2; the Sec. 5.2 fallback; and
the closed-form Test-1 equilibrium U_f = 59.55 km/s, T_f = 1.97 keV of Sec. 5.1.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle as O
from paper_2407_19151_gb300 import workloads as W


def cell_moments(st, m, species, rel=False, c=1.0):
    """Per cell: momentum (3), kinetic energy, and the scales sum m w |v| and sum KE."""
    cells = np.repeat(np.arange(st.n_cells), np.diff(st.offsets[:: st.n_species]))
    mp = np.asarray(m)[species] * st.w
    V = st.v()
    P = np.zeros((st.n_cells, 3))
    for d in range(3):
        np.add.at(P[:, d], cells, mp * V[:, d])
    v2 = (V ** 2).sum(1)
    ke = mp * v2 / (np.sqrt(1 + v2 / c ** 2) + 1) if rel else 0.5 * mp * v2
    E = np.zeros(st.n_cells)
    np.add.at(E, cells, ke)
    A = np.zeros(st.n_cells)
    np.add.at(A, cells, mp * np.sqrt(v2))
    return P, E, A


def make_state(wl):
    return O.State(wl.vx, wl.vy, wl.vz, wl.w, wl.offsets, wl.n_cells, wl.n_species)


@pytest.mark.parametrize("method", [O.TA77, O.N97])
@pytest.mark.parametrize("sort", [True, False])
def test_conservation_two_species(method, sort):
    wl = W.equilibration(n_cells=12, mean_count=24, precision="f64")
    st = make_state(wl)
    sp = wl.species_of_particles()
    P0, E0, A0 = cell_moments(st, wl.m, sp)
    p = O.Params(method=method, dt=wl.dt * 5, seed=wl.seed, sort_by_weight=sort)
    corr, fail = O.step(st, wl.q, wl.m, wl.lnL, p, n_steps=4)
    P1, E1, _ = cell_moments(st, wl.m, sp)
    assert fail.sum() == 0 and corr.sum() > 0
    assert np.max(np.abs(P1 - P0).max(axis=1) / A0) < 1e-13
    assert np.max(np.abs(E1 - E0) / E0) < 1e-13


def test_without_correction_conservation_is_only_statistical():
    # Sec. 5.1: unequal weights without the correction violate conservation at the percent level
    wl = W.equilibration(n_cells=12, mean_count=24, precision="f64")
    st = make_state(wl)
    sp = wl.species_of_particles()
    P0, E0, A0 = cell_moments(st, wl.m, sp)
    p = O.Params(method=O.N97, dt=wl.dt * 5, seed=wl.seed, correct=False)
    O.step(st, wl.q, wl.m, wl.lnL, p, n_steps=4)
    P1, E1, _ = cell_moments(st, wl.m, sp)
    assert np.max(np.abs(E1 - E0) / E0) > 1e-4


def test_momentum_shift_is_weight_biased():
    """Eq. vp_pm: v_pm = v_ps - B w_p with one B per cell, and sum m_p (v_pm - v_bs) = 0."""
    wl = W.equilibration(n_cells=6, mean_count=16, precision="f64")
    st = make_state(wl)
    sp = wl.species_of_particles()
    p = O.Params(method=O.N97, dt=wl.dt * 5, seed=3, max_corr_passes=0, fail_policy=O.FAIL_MOMENTUM_ONLY)
    bk = O.scatter(st, wl.q, wl.m, wl.lnL, 0, 1, 1, p)
    v_ps = st.v().copy()
    corr, fail = O.correct(st, wl.m, 0, 1, 1, p, bk)
    assert np.all(fail == 1) and corr.sum() == 0  # no energy pass allowed: every cell ends momentum-only
    v_pm = st.v()
    mp = wl.m[sp] * wl.w
    for c in range(wl.n_cells):
        a, b = wl.offsets[2 * c], wl.offsets[2 * c + 2]
        shift = v_ps[a:b] - v_pm[a:b]
        # least-squares B, then every particle's shift is B w_p up to the rounding of v_ps - B w_p
        B = (shift * wl.w[a:b, None]).sum(0) / (wl.w[a:b] ** 2).sum()
        resid = np.abs(shift - B * wl.w[a:b, None])
        assert np.all(resid <= 4 * np.spacing(np.abs(v_ps[a:b]).max()))
        assert np.abs(B).max() > 0
        dP = (mp[a:b, None] * (v_pm[a:b] - bk.T[a:b])).sum(0)
        assert np.abs(dP).max() < 1e-13 * (mp[a:b, None] * np.abs(v_pm[a:b])).sum()


def test_energy_partition_follows_eq_deltaes():
    wl = W.equilibration(n_cells=6, mean_count=40, precision="f64")
    sp = wl.species_of_particles()
    mp = wl.m[sp] * wl.w
    p_m = O.Params(method=O.N97, dt=wl.dt * 5, seed=4, max_corr_passes=0, fail_policy=O.FAIL_MOMENTUM_ONLY)
    st = make_state(wl)
    bk = O.scatter(st, wl.q, wl.m, wl.lnL, 0, 1, 1, p_m)
    st_full = O.State(st.vx, st.vy, st.vz, st.w, st.offsets, st.n_cells, 2)
    O.correct(st, wl.m, 0, 1, 1, p_m, bk)           # momentum only -> v_pm
    v_pm = st.v()
    p_f = O.Params(method=O.N97, dt=wl.dt * 5, seed=4)
    corr, fail = O.correct(st_full, wl.m, 0, 1, 1, p_f, bk)
    assert fail.sum() == 0
    v_f = st_full.v()
    ke = lambda v: 0.5 * mp * (v ** 2).sum(1)
    for c in range(wl.n_cells):
        sl = [slice(wl.offsets[2 * c + s], wl.offsets[2 * c + s + 1]) for s in (0, 1)]
        E_bs = sum(ke(bk.T)[x].sum() for x in sl)
        E_pm = [ke(v_pm)[x].sum() for x in sl]
        dE = sum(E_pm) - E_bs
        wbar = [wl.w[x].mean() for x in sl]
        dEa = wbar[0] * E_pm[0] / (wbar[0] * E_pm[0] + wbar[1] * E_pm[1]) * dE
        absorbed_a = E_pm[0] - ke(v_f)[sl[0]].sum()
        assert absorbed_a == pytest.approx(dEa, rel=1e-9, abs=1e-14 * E_bs)


def test_energy_pair_exact_and_first_order():
    rng = np.random.default_rng(8)
    for _ in range(50):
        m1, m2 = rng.uniform(0.5, 5, 2)
        v1, v2 = rng.normal(size=3), rng.normal(size=3)
        K = O.pair_kecm(False, 1.0, m1, m2, v1, v2)
        assert K == pytest.approx(0.5 * m1 * m2 / (m1 + m2) * np.sum((v1 - v2) ** 2), rel=1e-15)
        for U in [0.03 * K, -0.05 * K, 1e-9 * K]:
            a, b = O.energy_pair(False, 1.0, m1, m2, v1, v2, U)
            np.testing.assert_allclose(m1 * a + m2 * b, m1 * v1 + m2 * v2, rtol=0, atol=1e-14)
            dke = 0.5 * m1 * (a @ a) + 0.5 * m2 * (b @ b) - 0.5 * m1 * (v1 @ v1) - 0.5 * m2 * (v2 @ v2)
            KE = 0.5 * m1 * (v1 @ v1) + 0.5 * m2 * (v2 @ v2)
            assert dke == pytest.approx(-U, rel=1e-9, abs=1e-15 * KE)
            # zero-angle: the relative velocity keeps its direction
            vr, vrp = v1 - v2, a - b
            assert np.linalg.norm(np.cross(vr, vrp)) < 1e-13 * np.linalg.norm(vr) ** 2
    # Eqs. vp1_inelastic_2 / vp2_inelastic_2: m1 = m2, U = -fE K  ->  dv1 ~ +(fE/4)(v1 - v2)
    v1, v2 = np.array([1.0, 0.2, -0.3]), np.array([-0.4, 0.5, 0.1])
    for fE in [1e-2, 1e-3]:
        K = O.pair_kecm(False, 1.0, 1.0, 1.0, v1, v2)
        a, b = O.energy_pair(False, 1.0, 1.0, 1.0, v1, v2, -fE * K)
        np.testing.assert_allclose(a - v1, fE / 4 * (v1 - v2), rtol=fE)
        np.testing.assert_allclose(b - v2, -fE / 4 * (v1 - v2), rtol=fE)


def test_relativistic_energy_pair_solves_eq_alpha_eq0():
    rng = np.random.default_rng(9)
    c = 1.0
    for _ in range(200):
        m1, m2 = rng.uniform(0.5, 3, 2)
        u1 = rng.normal(size=3) * rng.choice([1e-3, 0.1, 3.0])
        u2 = rng.normal(size=3) * rng.choice([1e-3, 0.1, 3.0])
        K = O.pair_kecm(True, c, m1, m2, u1, u2)
        E = lambda m, u: m * c * c * math.sqrt(1 + u @ u / c ** 2)
        # KE_cm = E_cm - (m1 + m2) c^2 with E_cm^2 = E_tot^2 - |p_tot|^2 c^2 (checked in 40-digit arithmetic)
        import mpmath
        with mpmath.workdps(40):
            Et = sum(mpmath.mpf(m) * mpmath.sqrt(1 + sum(mpmath.mpf(x) ** 2 for x in u)) for m, u in ((m1, u1), (m2, u2)))
            pt = [mpmath.mpf(m1) * mpmath.mpf(a) + mpmath.mpf(m2) * mpmath.mpf(b) for a, b in zip(u1, u2)]
            Kref = float(mpmath.sqrt(Et ** 2 - sum(x ** 2 for x in pt)) - m1 - m2)
        assert K == pytest.approx(Kref, rel=1e-10)
        for U in [0.04 * K, -0.05 * K]:
            a, b = O.energy_pair(True, c, m1, m2, u1, u2, U)
            np.testing.assert_allclose(m1 * a + m2 * b, m1 * u1 + m2 * u2, rtol=0,
                                       atol=1e-14 * (m1 * np.abs(u1).max() + m2 * np.abs(u2).max()))
            Etot = E(m1, u1) + E(m2, u2)
            assert E(m1, a) + E(m2, b) - Etot == pytest.approx(-U, rel=1e-7, abs=1e-14 * Etot)
    # c -> infinity reduces to the non-relativistic pair
    u1, u2 = np.array([0.3, 0.1, -0.2]), np.array([-0.1, 0.2, 0.4])
    for U in [0.02, -0.03]:
        K = O.pair_kecm(False, 1.0, 2.0, 3.0, u1, u2)
        a, b = O.energy_pair(True, 1e5, 2.0, 3.0, u1, u2, U * K)
        an, bn = O.energy_pair(False, 1.0, 2.0, 3.0, u1, u2, U * K)
        np.testing.assert_allclose(a, an, rtol=1e-8)
        np.testing.assert_allclose(b, bn, rtol=1e-8)


def test_relativistic_step_conserves():
    wl = W.relativistic_beam(n_cells=10, count_lo=16, count_hi=64, precision="f64")
    st = make_state(wl)
    sp = wl.species_of_particles()
    P0, E0, A0 = cell_moments(st, wl.m, sp, rel=True)
    p = O.Params(method=O.N97, relativistic=True, dt=wl.dt * 5, seed=wl.seed, c=wl.c)
    corr, fail = O.step(st, wl.q, wl.m, wl.lnL, p, n_steps=3)
    P1, E1, _ = cell_moments(st, wl.m, sp, rel=True)
    # cells whose correction failed were rolled back interaction by interaction, so every cell conserves
    assert fail.sum() < wl.n_cells * 3 * len(wl.interactions()) // 2 and corr.sum() > 0
    assert np.max(np.abs(P1 - P0).max(axis=1) / A0) < 1e-13
    assert np.max(np.abs(E1 - E0) / E0) < 1e-13


def test_equal_weights_correction_is_noop():
    wl = W.isotropisation(n_cells=6, per_cell=32)
    wl.w[:] = 3.0
    a, b = make_state(wl), make_state(wl)
    O.step(a, wl.q, wl.m, wl.lnL, O.Params(method=O.N97, dt=wl.dt, seed=2, correct=True), n_steps=3)
    O.step(b, wl.q, wl.m, wl.lnL, O.Params(method=O.N97, dt=wl.dt, seed=2, correct=False), n_steps=3)
    scale = np.sqrt((a.v() ** 2).sum(1)).max()
    assert np.abs(a.v() - b.v()).max() < 1e-13 * scale


def test_failure_rollback_and_momentum_only():
    """Sec. 5.2: three particles, one weight 1e6 times the others; the heavy one scatters and the energy error
    cannot be re-absorbed. Rollback restores the pre-scatter velocities; momentum-only keeps momentum."""
    v = np.array([[1.0, 0.0, 0.0], [-0.5, 0.3, 0.0], [0.0, -0.4, 0.7]])
    w = np.array([1e6, 1.0, 1.0])
    found = None
    for seed in range(200):
        st = O.State(v[:, 0], v[:, 1], v[:, 2], w, np.array([0, 3]), 1, 1)
        p = O.Params(method=O.N97, dt=0.5, seed=seed)
        corr, fail = O.step(st, [-1.0], [1.0], 10.0, p)
        if fail[0]:
            found = seed
            np.testing.assert_array_equal(st.v(), v)  # rolled back
            break
    assert found is not None
    st = O.State(v[:, 0], v[:, 1], v[:, 2], w, np.array([0, 3]), 1, 1)
    p = O.Params(method=O.N97, dt=0.5, seed=found, fail_policy=O.FAIL_MOMENTUM_ONLY)
    corr, fail = O.step(st, [-1.0], [1.0], 10.0, p)
    assert fail[0] == 1
    P0, P1 = (w[:, None] * v).sum(0), (w[:, None] * st.v()).sum(0)
    assert np.abs(P1 - P0).max() < 1e-13 * (w[:, None] * np.abs(v)).sum()
    assert not np.array_equal(st.v(), v)


def test_correction_pairs_fall_with_fE():
    counts = []
    for fE in [0.02, 0.05, 0.2]:
        wl = W.equilibration(n_cells=8, mean_count=64, precision="f64")
        st = make_state(wl)
        corr, fail = O.step(st, wl.q, wl.m, wl.lnL, O.Params(method=O.N97, dt=wl.dt * 5, seed=1, fE=fE), 2)
        assert fail.sum() <= 1
        counts.append(corr.sum())
    assert counts[0] > counts[1] > counts[2]


# ------------------------------------------------------------------------------------------ Test 1, Sec. 5.1
E_CH = 1.602176634e-19
M_E = 9.1093837015e-31
M_U = 1.66053906660e-27
EPS0 = 8.8541878128e-12


GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


def paper_test1_equilibrium():
    """Conservation of the T1 populations (n_A = 1e19/cc, U_A = 655 km/s, T = 500 eV; n_B = 1e20/cc at rest)."""
    g = GOLDEN["test1"]
    mi = g["A_mass_number"] * M_U - g["Z"] * M_E
    nA, nB, UA, T = g["n_A_per_cc"], g["n_B_per_cc"], g["U_A_km_s"] * 1e3, g["T_A_eV"]
    Uf = UA * nA / (nA + nB)
    # 3/2 (nA + nB) Tf + 1/2 m (nA + nB) Uf^2 = 3/2 (nA + nB) T + 1/2 m nA UA^2
    Tf = T + (0.5 * mi * nA * UA ** 2 - 0.5 * mi * (nA + nB) * Uf ** 2) / (1.5 * (nA + nB)) / E_CH
    return Uf, Tf


def test_test1_closed_form():
    Uf, Tf = paper_test1_equilibrium()
    assert Uf / 1e3 == pytest.approx(GOLDEN["test1"]["U_f_km_s"], abs=0.005)
    assert Tf / 1e3 == pytest.approx(GOLDEN["test1"]["T_f_keV"], abs=0.005)


def test_test3_closed_form():
    """Sec. 5.3: energy conservation of the e / C6+ plasma fixes the common final temperature at 136 eV, and the
    quoted time step is of order 1/100 of tau_e."""
    g = GOLDEN["test3"]
    Tf = (g["n_e_per_cc"] * g["T_e_eV"] + g["n_i_per_cc"] * g["T_i_eV"]) / (g["n_e_per_cc"] + g["n_i_per_cc"])
    assert Tf == pytest.approx(g["T_f_eV"], abs=0.5)
    tau_e = g["tau_e_prefactor"] * g["T_e_eV"] ** 1.5 / (g["Z"] * g["n_e_per_cc"] * g["lnLambda"])
    assert 50 < tau_e / (g["dt_fs"] * 1e-15) < 300


def test_test1_relaxes_to_closed_form():
    """Scaled T1b (40 + 40 particles per cell, w_A : w_B = 1 : 10, SI units, dt = 50 fs, lnL = 10, N97): per-cell
    populations are given exactly the nominal mean velocity and temperature, so conservation fixes the
    equilibrium at the closed form; the oracle must conserve it to round-off and relax to it."""
    mi, q = 12 * M_U - 6 * M_E, 6 * E_CH
    nA, nB, UA, T = 1e25, 1e26, 655e3, 500.0 * E_CH
    NA = NB = 40
    ncell, dV = 8, 1e-21
    wA, wB = nA * dV / NA, nB * dV / NB
    rng = np.random.default_rng(0)

    def population(n, U):
        x = rng.normal(size=(n, 3))
        x -= x.mean(0)
        x *= np.sqrt(3 * T / mi / (x ** 2).sum(1).mean())
        x[:, 0] += U
        return x

    v = np.vstack([np.vstack([population(NA, UA), population(NB, 0.0)]) for _ in range(ncell)])
    w = np.tile(np.r_[np.full(NA, wA), np.full(NB, wB)], ncell)
    pop = np.tile(np.r_[np.zeros(NA), np.ones(NB)], ncell).astype(bool)
    off = np.arange(ncell + 1, dtype=np.int64) * (NA + NB)
    st = O.State(v[:, 0], v[:, 1], v[:, 2], w, off, ncell, 1)
    P0, E0 = (mi * w * v[:, 0]).sum(), (0.5 * mi * w * (v ** 2).sum(1)).sum()
    p = O.Params(method=O.N97, dt=50e-15, dV=dV, eps0=EPS0, fE=0.05, seed=7)
    corr, fail = O.step(st, [q], [mi], 10.0, p, n_steps=4000)
    # equilibrium phase: time-average the population moments over 8 samples 500 steps apart
    Uf, Tf = paper_test1_equilibrium()
    samples = []
    for k in range(8):
        p.step += 4000 if k == 0 else 500
        c2, f2 = O.step(st, [q], [mi], 10.0, p, n_steps=500)
        fail = fail + f2
        V = st.v()
        row = []
        for sel in (pop, ~pop):
            U = (w[sel, None] * V[sel]).sum(0) / w[sel].sum()
            Tp = mi * (w[sel] * ((V[sel] - U) ** 2).sum(1)).sum() / (3 * w[sel].sum()) / E_CH
            row += [U[0], Tp]
        samples.append(row)
        assert abs((mi * w * V[:, 0]).sum() - P0) < 1e-12 * abs(P0)
        assert abs((0.5 * mi * w * (V ** 2).sum(1)).sum() - E0) < 1e-12 * E0
    assert fail.sum() == 0
    UB, TB, UA_, TA_ = np.mean(samples, axis=0)
    assert UB == pytest.approx(Uf, rel=0.03) and UA_ == pytest.approx(Uf, rel=0.1)
    assert TB == pytest.approx(Tf, rel=0.03) and TA_ == pytest.approx(Tf, rel=0.05)


def test_oracle_resume_is_bit_exact():
    """Checkpoint / resume on the oracle: four steps equal two steps, a saved copy of the state, then two more
    steps from step + 2 (every draw is keyed by the step index)."""
    wl = W.three_species(n_cells=12, mean_count=60, precision="f64")
    p = O.Params(method=wl.method, dt=wl.dt * 3, seed=wl.seed, step=40)
    a = O.State(wl.vx, wl.vy, wl.vz, wl.w, wl.offsets, wl.n_cells, wl.n_species)
    O.step(a, wl.q, wl.m, wl.lnL, p, n_steps=4)
    b = O.State(wl.vx, wl.vy, wl.vz, wl.w, wl.offsets, wl.n_cells, wl.n_species)
    O.step(b, wl.q, wl.m, wl.lnL, p, n_steps=2)
    saved = b.v().copy()
    c = O.State(saved[:, 0], saved[:, 1], saved[:, 2], wl.w, wl.offsets, wl.n_cells, wl.n_species)
    O.step(c, wl.q, wl.m, wl.lnL, O.Params(method=wl.method, dt=wl.dt * 3, seed=wl.seed, step=42), n_steps=2)
    np.testing.assert_array_equal(a.v(), c.v())
