"""Pins of the oracle gradient (central differences of the oracle step, decisions fixed). Every interaction conserves
the momentum and the kinetic energy of its cell exactly (Eq. vp_pm, Eq. Econs), so along the cotangents
cot_p = m_p w_p e_x and cot_p = m_p w_p v_p(final) the derivative has a closed form:
  momentum:  dL/dv_p,x = m_p w_p,  dL/dv_p,y = 0,  dL/dw_p = m_p (v_p,x(initial) - v_p,x(final)),  dL/dlnL = 0;
  energy:    dL/dv_p = m_p w_p v_p(initial),  dL/dw_p = m_p (|v_p(initial)|^2 - |v_p(final)|^2) / 2,  dL/dlnL = 0.
(L uses the nominal weights in the cotangent, hence the final-velocity terms in dL/dw.)"""
import numpy as np
import pytest

import oracle as O
from oracle import gradient as G
from paper_2407_19151_gb300 import workloads as W


def _case(method):
    wl = W.differentiable(n_cells=3, per_species=12)
    wl.method = method
    p = O.Params(method=method, dt=wl.dt * 20, fE=wl.fE, seed=wl.seed, step=3)
    return wl, p


def _args(wl):
    return (wl.offsets, wl.n_cells, wl.n_species, wl.q, wl.m, wl.lnL)


@pytest.mark.parametrize("method", [O.TA77, O.N97])
def test_fd_gradient_of_momentum_and_energy(method):
    wl, p = _case(method)
    v0 = wl.vx[:, None] * [1, 0, 0] + wl.vy[:, None] * [0, 1, 0] + wl.vz[:, None] * [0, 0, 1]
    sp = wl.species_of_particles()
    mp = wl.m[sp]
    vf, corr, fail = G.forward(v0, wl.w, *_args(wl), p, 2)
    assert corr.sum() > 0 and fail.sum() == 0  # the correction did work in these cells
    rng = np.random.default_rng(0)
    cot_p = np.zeros_like(v0)
    cot_p[:, 0] = mp * wl.w
    cot_e = (mp * wl.w)[:, None] * vf
    checked = 0
    for idx in rng.choice(wl.n, 6, replace=False):
        for cot, want_v, want_w in (
                (cot_p, [mp[idx] * wl.w[idx], 0.0, 0.0], mp[idx] * (v0[idx, 0] - vf[idx, 0])),
                (cot_e, mp[idx] * wl.w[idx] * v0[idx], 0.5 * mp[idx] * (v0[idx] @ v0[idx] - vf[idx] @ vf[idx]))):
            scale_v = mp[idx] * wl.w[idx] * max(np.abs(v0[idx]).max(), 1.0)
            for d in range(3):
                g, g2, same = G.fd_derivative(cot, v0, wl.w, *_args(wl), p, 2, ("v", int(idx), d))
                if not same or abs(g - g2) > 1e-6 * scale_v:
                    continue
                assert abs(g - want_v[d]) <= 1e-6 * scale_v, (idx, d, g, want_v[d])
                checked += 1
            g, g2, same = G.fd_derivative(cot, v0, wl.w, *_args(wl), p, 2, ("w", int(idx)))
            sw = mp[idx] * max(v0[idx] @ v0[idx], vf[idx] @ vf[idx], 1.0)
            if same and abs(g - g2) <= 1e-6 * sw:
                assert abs(g - want_w) <= 1e-6 * sw, (idx, g, want_w)
                checked += 1
    for cot, scale in ((cot_p, np.abs(cot_p).sum()), (cot_e, np.abs(cot_e * v0).sum())):
        g, g2, same = G.fd_derivative(cot, v0, wl.w, *_args(wl), p, 2, ("lnL", 0, 1))
        assert abs(g) <= 1e-7 * scale
    assert checked >= 30


def test_fd_gradient_detects_a_dropped_term():
    """A gradient that ignores the moment correction (scatter only) breaks the momentum closed form: the check above
    is sensitive to it."""
    wl, p = _case(O.N97)
    v0 = np.stack([wl.vx, wl.vy, wl.vz], axis=1)
    sp = wl.species_of_particles()
    mp = wl.m[sp]
    cot = np.zeros_like(v0)
    cot[:, 0] = mp * wl.w
    pn = O.Params(**{**p.__dict__, "correct": False})
    worst = 0.0
    for idx in range(0, wl.n, 7):
        g, _, _ = G.fd_derivative(cot, v0, wl.w, *_args(wl), pn, 2, ("w", int(idx)))
        vf, _, _ = G.forward(v0, wl.w, *_args(wl), pn, 2)
        worst = max(worst, abs(g - mp[idx] * (v0[idx, 0] - vf[idx, 0])) / (mp[idx] * np.abs(v0[idx]).max()))
    assert worst > 1e-3
