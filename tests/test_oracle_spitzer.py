"""Physics integration pin of the oracle: electron-ion temperature relaxation against the 0D Spitzer model
(Eq. 0DSpitzer, Sec. 5.3: dT_e/dt = -nu_T (T_e - T_i), dT_i/dt = -Z dT_e/dt with n_e = Z n_i).

The rate used is Spitzer's for Maxwellians of any mass ratio,
    nu = 8 sqrt(2 pi) n q_e^2 q_i^2 lnL sqrt(m_e m_i) / (3 (4 pi eps0)^2 (m_e T_i + m_i T_e)^{3/2}),
which reduces to the paper's nu_T = 2 m_e / M_i / tau_e for M_i >> m_e, and which the small-angle binary model
reproduces exactly for Maxwellians (the Gaussian average E[(mu/m_e - alpha) / |u|] of the pair drag).

Measured behaviour of the binary method, which the bounds encode: with N97 at nu dt = 0.02 the angle saturation
(1 - exp(-s) instead of s for slow pairs) lowers the rate by ~4%; with the physical self-collision rates the
electron distribution is not kept quite Maxwellian at mass ratio 25 (the exchange is dominated by slow electrons),
which lowers it by ~9% more; with ten times the self-collision rate the relaxation runs at 0.93 +- 0.02 of the
Spitzer rate. A factor of two anywhere in the e-i scattering length, a wrong reduced mass or a lost weight factor
moves the ratio far outside [0.87, 0.99]."""
import math

import numpy as np

import oracle as O


def _relaxed_fraction(seed, C=64, N=256, M=25.0, steps=250, nu_dt=0.02, self_boost=10.0):
    rng = np.random.default_rng(seed)
    Te0, Ti0, lnL = 1.0, 0.25, 10.0
    # weighted particles, equal densities (Z = 1): log-uniform weights rescaled per cell so that n_i = n_e
    we = 10.0 ** rng.uniform(0, 1, (C, N))
    wi = 10.0 ** rng.uniform(0, 1, (C, N))
    wi *= we.sum(1, keepdims=True) / wi.sum(1, keepdims=True)
    n = float(we.sum(1).mean())
    ve = rng.normal(0, math.sqrt(Te0), (C, N, 3))
    vi = rng.normal(0, math.sqrt(Ti0 / M), (C, N, 3))
    v = np.concatenate([ve, vi], axis=1).reshape(-1, 3)
    w = np.concatenate([we, wi], axis=1).reshape(-1)
    off = np.zeros(2 * C + 1, np.int64)
    off[1:] = np.cumsum(np.tile([N, N], C))
    dt = nu_dt / (lnL * n / (4 * math.pi * Te0 ** 1.5))
    q, m = np.array([-1.0, 1.0]), np.array([1.0, M])
    L = np.array([[lnL * self_boost, lnL], [lnL, lnL * self_boost]])
    sp = np.tile(np.r_[np.zeros(N, int), np.ones(N, int)], C)

    def temps(x):
        out = []
        for s in (0, 1):
            sel = sp == s
            ws, xs = w[sel], x[sel]
            V = (ws[:, None] * xs).sum(0) / ws.sum()
            out.append(m[s] * (ws * ((xs - V) ** 2).sum(1)).sum() / (3 * ws.sum()))
        return out

    def rates(Te, Ti):
        k = 8 * math.sqrt(2 * math.pi) * n * lnL * math.sqrt(m[0] * m[1]) / (
            3 * (4 * math.pi) ** 2 * (m[0] * Ti + m[1] * Te) ** 1.5)
        return k * (Ti - Te), k * (Te - Ti)

    st = O.State(v[:, 0].copy(), v[:, 1].copy(), v[:, 2].copy(), w, off, C, 2)
    T0 = temps(st.v())
    O.step(st, q, m, L, O.Params(method=O.N97, dt=dt, seed=100 + seed, step=0, fE=0.05), n_steps=steps)
    Te, Ti = temps(st.v())
    T = list(T0)
    for _ in range(4 * steps):  # RK4 on the Spitzer ODE
        h = dt / 4
        a = rates(*T)
        b = rates(T[0] + h / 2 * a[0], T[1] + h / 2 * a[1])
        c = rates(T[0] + h / 2 * b[0], T[1] + h / 2 * b[1])
        d = rates(T[0] + h * c[0], T[1] + h * c[1])
        T = [T[i] + h / 6 * (a[i] + 2 * b[i] + 2 * c[i] + d[i]) for i in range(2)]
    # energy conservation of the corrected method: n_e T_e + n_i T_i unchanged
    assert abs((Te + Ti) - (T0[0] + T0[1])) < 1e-9 * (T0[0] + T0[1]) + 5e-3
    d0 = T0[0] - T0[1]
    return (d0 - (Te - Ti)) / (d0 - (T[0] - T[1]))


def test_electron_ion_relaxation_follows_spitzer():
    r = [_relaxed_fraction(s) for s in range(3)]
    assert 0.87 < float(np.mean(r)) < 0.99, r
