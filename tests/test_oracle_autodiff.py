"""Pins of the reverse-mode oracle gradient (oracle/autodiff.py: the step transcribed in PyTorch CPU FP64 and
differentiated by autograd, decisions held fixed). Its forward must equal the C oracle's step to rounding (so the
transcription takes the same decisions and computes the same function); its gradient must satisfy, for every
particle, the closed forms that exact momentum and energy conservation of every interaction fix (the cotangents
m w e_x and m w v_final, see tests/test_oracle_gradient.py), and must equal central differences of the C oracle
(a different method on a different implementation) on sampled entries."""
import numpy as np
import pytest

import oracle as O
from oracle import autodiff as AD
from oracle import gradient as G
from paper_2407_19151_gb300 import workloads as W


def _even(method):
    wl = W.differentiable(n_cells=4, per_species=12)
    return wl, O.Params(method=method, dt=wl.dt * 20, fE=wl.fE, seed=wl.seed, step=3)


def _poisson(method):
    """Odd intra-species counts (the triplet), populations of 0 and 1 (interactions skipped or one-sided energy
    partition)."""
    wl = W.equilibration(n_cells=12, mean_count=5, precision="f64", method=method)
    assert (wl.counts % 2 == 1).any() and (wl.counts < 2).any()
    return wl, O.Params(method=method, dt=wl.dt * 5, fE=wl.fE, seed=wl.seed, step=3)


def _failing(method):
    """A cap fraction so small that some energy loops run out of passes: the rollback of Sec. 5.2."""
    wl = W.differentiable(n_cells=6, per_species=10)
    return wl, O.Params(method=method, dt=wl.dt * 40, fE=1e-4, max_corr_passes=2, seed=wl.seed, step=5)


def _v0(wl):
    return np.stack([wl.vx, wl.vy, wl.vz], axis=1).astype(np.float64)


def _args(wl):
    return (wl.offsets, wl.n_cells, wl.n_species, wl.q, wl.m)


CASES = {"even": _even, "poisson": _poisson, "failing": _failing}


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("method", [O.TA77, O.N97])
def test_autodiff_forward_equals_oracle(method, case):
    import torch
    wl, p = CASES[case](method)
    v = AD.step(torch.tensor(_v0(wl)), torch.tensor(wl.w), torch.tensor(np.asarray(wl.lnL, dtype=np.float64)),
                wl.offsets, wl.n_cells, wl.n_species, wl.q, wl.m, p, n_steps=2).numpy()
    st = O.State(wl.vx, wl.vy, wl.vz, wl.w, wl.offsets, wl.n_cells, wl.n_species)
    corr, fail = O.step(st, wl.q, wl.m, wl.lnL, p, n_steps=2)
    ref = st.v()
    assert np.abs(v - ref).max() <= 1e-13 * np.abs(ref).max()
    if case == "failing":
        assert fail.sum() > 0
    else:
        assert corr.sum() > 0


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("method", [O.TA77, O.N97])
def test_autodiff_gradient_closed_forms(method, case):
    """Every particle: momentum and energy cotangents give the conservation closed forms for dL/dv and dL/dw, and
    dL/dlnL = 0."""
    wl, p = CASES[case](method)
    v0 = _v0(wl)
    sp = wl.species_of_particles()
    mp = wl.m[sp]
    mw = mp * wl.w
    cot = np.zeros_like(v0)
    cot[:, 0] = mw
    vf, gv, gw, gL = AD.gradient(cot, v0, wl.w, wl.lnL, *_args(wl), p, 2)
    want = np.zeros_like(v0)
    want[:, 0] = mw
    scale = mw * np.maximum(np.abs(v0).max(1), np.abs(vf).max(1))
    assert (np.abs(gv - want).max(1) / mw).max() < 1e-10
    assert (np.abs(gw - mp * (v0[:, 0] - vf[:, 0])) * wl.w / scale).max() < 1e-10
    assert np.abs(gL).max() < 1e-10 * np.abs(mw[:, None] * vf).sum()
    vf, gv, gw, gL = AD.gradient(mw[:, None] * vf, v0, wl.w, wl.lnL, *_args(wl), p, 2)
    e0, ef = (v0 ** 2).sum(1), (vf ** 2).sum(1)
    escale = mw * np.maximum(e0, ef)
    assert (np.abs(gv - mw[:, None] * v0).max(1) * np.abs(v0).max(1) / escale).max() < 1e-10
    assert (np.abs(gw - 0.5 * mp * (e0 - ef)) * wl.w / escale).max() < 1e-10
    assert np.abs(gL).max() < 1e-10 * (mw * ef).sum()


@pytest.mark.parametrize("case", ["even", "poisson"])
@pytest.mark.parametrize("method", [O.TA77, O.N97])
def test_autodiff_gradient_equals_finite_differences(method, case):
    """A random cotangent: sampled dL/dv, dL/dw and every dL/dlnL against central differences of the C oracle (a
    sample whose quotients at h and h/2 disagree straddles a decision and is skipped)."""
    wl, p = CASES[case](method)
    v0 = _v0(wl)
    rng = np.random.default_rng(21)
    cot = rng.standard_normal(v0.shape)
    _, gv, gw, gL = AD.gradient(cot, v0, wl.w, wl.lnL, *_args(wl), p, 2)
    args = (wl.offsets, wl.n_cells, wl.n_species, wl.q, wl.m, wl.lnL, p, 2)
    checked = 0
    for idx in rng.choice(wl.n, 8, replace=False):
        idx = int(idx)
        for d in range(3):
            g, g2, same = G.fd_derivative(cot, v0, wl.w, *args, ("v", idx, d))
            tol = 1e-6 * max(abs(g), np.abs(cot).max())
            if same and abs(g - g2) <= tol:
                assert abs(gv[idx, d] - g) <= tol, (idx, d, gv[idx, d], g)
                checked += 1
        seg = np.searchsorted(wl.offsets, idx, side="right") - 1
        if np.count_nonzero(wl.w[wl.offsets[seg]:wl.offsets[seg + 1]] == wl.w[idx]) > 1:
            continue  # a weight tied with another of its population: w_max and the weight order are not smooth
        g, g2, same = G.fd_derivative(cot, v0, wl.w, *args, ("w", idx))
        tol = 1e-6 * max(abs(g), np.abs(cot).max() * np.abs(v0).max() / wl.w[idx])
        if same and abs(g - g2) <= tol:
            assert abs(gw[idx] - g) <= tol, (idx, gw[idx], g)
            checked += 1
    for a, b in ((0, 0), (0, 1), (1, 1)):
        g, g2, same = G.fd_derivative(cot, v0, wl.w, *args, ("lnL", a, b))
        tol = 1e-6 * max(abs(g), 1e-3 * np.abs(cot * v0).sum() / wl.lnL[a, b])
        if same and abs(g - g2) <= tol:
            assert abs(gL[a, b] + (gL[b, a] if a != b else 0.0) - g) <= tol, (a, b, gL[a, b], g)
            checked += 1
    assert checked >= 20


def test_autodiff_detects_a_wrong_angle_derivative(monkeypatch):
    """Planted mistake: doubling dA/ds of the N97 root moves sampled entries away from the finite differences, so
    the comparison above would catch an error there."""
    wl, p = _even(O.N97)
    v0 = _v0(wl)
    cot = np.random.default_rng(2).standard_normal(v0.shape)
    _, gv, _, _ = AD.gradient(cot, v0, wl.w, wl.lnL, *_args(wl), p, 2)
    real = AD._n97_dL
    monkeypatch.setattr(AD, "_n97_dL", lambda A: 0.5 * real(A))
    _, gv_bad, _, _ = AD.gradient(cot, v0, wl.w, wl.lnL, *_args(wl), p, 2)
    assert np.abs(gv_bad - gv).max() > 1e-4 * np.abs(gv).max()
