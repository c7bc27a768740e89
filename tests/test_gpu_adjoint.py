"""GPU parity of the pathwise adjoint (mcc_adjoint, collision_steps) against the oracle: its recomputed forward
against the oracle step, its gradients against the closed forms that exact momentum and energy conservation fix,
against the reverse-mode oracle gradient (oracle/autodiff.py) entry by entry over every particle, and against
central differences of the oracle step on the same seed."""
import numpy as np
import pytest

import oracle as O
from oracle import autodiff as AD
from oracle import gradient as G
from paper_2407_19151_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mcc():
    import paper_2407_19151_gb300 as m
    m.build()
    return m


def _tensors(wl):
    import torch
    v = [torch.tensor(np.asarray(x, dtype=np.float64), device="cuda") for x in (wl.vx, wl.vy, wl.vz)]
    w = torch.tensor(wl.w, dtype=torch.float64, device="cuda")
    off = torch.tensor(wl.offsets, device="cuda")
    L = torch.tensor(np.asarray(wl.lnL, dtype=np.float64))
    return v, w, off, L


def _case(method, n_cells=3, per_species=12, dt_scale=20):
    wl = W.differentiable(n_cells=n_cells, per_species=per_species)
    wl.method = method
    kw = dict(method=method, dt=wl.dt * dt_scale, fE=wl.fE, seed=wl.seed, step=3)
    return wl, kw


@pytest.mark.parametrize("method", [W.TA77, W.N97])
def test_adjoint_forward_matches_oracle(mcc, method):
    import torch
    wl, kw = _case(method, n_cells=24, per_species=40)
    v, w, off, _ = _tensors(wl)
    p = mcc.Params(**kw)
    sp = list(zip(wl.q.tolist(), wl.m.tolist()))
    mc = int(wl.counts.sum(1).max())
    for k, (a, b) in enumerate(mcc.default_interactions(wl.n_species)):
        out = [torch.empty_like(x) for x in v]
        mcc.mcc_adjoint(*v, w, off, wl.n_cells, wl.n_species, sp, wl.lnL, a, b, k, p, mc, out=out)
        v = out
    mcc.sync_status(0)
    st = O.State(wl.vx, wl.vy, wl.vz, wl.w, wl.offsets, wl.n_cells, wl.n_species)
    O.step(st, wl.q, wl.m, wl.lnL, O.Params(**kw))
    got = np.stack([x.cpu().numpy() for x in v], axis=1)
    ref = st.v()
    scale = np.sqrt((ref ** 2).sum(1).mean())
    assert np.abs(got - ref).max() / scale < 1e-12


def _grads(mcc, wl, kw, cot_fn, n_steps=2, every=10, tape=False):
    import torch
    v, w, off, L = _tensors(wl)
    for x in (*v, w, L):
        x.requires_grad_(True)
    sp = list(zip(wl.q.tolist(), wl.m.tolist()))
    out = mcc.collision_steps(*v, w, L, off, wl.n_cells, wl.n_species, sp, mcc.Params(**kw), n_steps,
                              checkpoint_every=every, tape=tape)
    vf = np.stack([x.detach().cpu().numpy() for x in out], axis=1)
    cot = torch.tensor(cot_fn(vf), device="cuda")
    loss = sum((cot[:, d] * out[d]).sum() for d in range(3))
    loss.backward()
    gv = np.stack([x.grad.cpu().numpy() for x in v], axis=1)
    return vf, gv, w.grad.cpu().numpy(), L.grad.numpy()


def _poisson_case(method):
    """Poisson counts (odd intra counts run the triplet, small and empty populations skip interactions)."""
    wl = W.equilibration(n_cells=40, mean_count=5, precision="f64", method=method)
    assert (wl.counts % 2 == 1).any() and (wl.counts < 2).any()
    return wl, dict(method=method, dt=wl.dt * 5, fE=wl.fE, seed=wl.seed, step=3)


@pytest.mark.parametrize("case", ["even", "poisson"])
@pytest.mark.parametrize("method", [W.TA77, W.N97])
def test_adjoint_conservation_closed_forms(mcc, method, case):
    """Momentum: cot = m w e_x gives dL/dv = m w e_x, dL/dw = m (v0_x - vf_x), dL/dlnL = 0. Energy: cot = m w vf gives
    dL/dv = m w v0, dL/dw = m (|v0|^2 - |vf|^2)/2, dL/dlnL = 0 (every particle, not a sample)."""
    wl, kw = _case(method, n_cells=16, per_species=64) if case == "even" else _poisson_case(method)
    sp = wl.species_of_particles()
    mw = wl.m[sp] * wl.w
    v0 = np.stack([wl.vx, wl.vy, wl.vz], axis=1)

    def cot_p(vf):
        c = np.zeros_like(vf)
        c[:, 0] = mw
        return c

    vf, gv, gw, gL = _grads(mcc, wl, kw, cot_p)
    scale = mw * np.maximum(np.abs(v0).max(1), np.abs(vf).max(1))
    want = np.zeros_like(v0)
    want[:, 0] = mw
    assert (np.abs(gv - want).max(1) / mw).max() < 1e-9
    assert (np.abs(gw - wl.m[sp] * (v0[:, 0] - vf[:, 0])) * wl.w / scale).max() < 1e-9
    assert np.abs(gL).max() < 1e-9 * np.abs(mw[:, None] * vf).sum()

    vf, gv, gw, gL = _grads(mcc, wl, kw, lambda vf: mw[:, None] * vf)
    e0 = (v0 ** 2).sum(1)
    ef = (vf ** 2).sum(1)
    escale = mw * np.maximum(e0, ef)
    assert (np.abs(gv - mw[:, None] * v0).max(1) * np.abs(v0).max(1) / escale).max() < 1e-9
    assert (np.abs(gw - 0.5 * wl.m[sp] * (e0 - ef)) * wl.w / escale).max() < 1e-9
    assert np.abs(gL).max() < 1e-9 * (mw * ef).sum()


@pytest.mark.parametrize("tape", [False, True], ids=["checkpoints", "tape"])
def test_adjoint_conservation_closed_forms_full_size(mcc, tape):
    """The differentiable workload at full size (1024 cells x 512, two species, N97, FP64) over its 50 steps with a
    checkpoint every 10 (or recorded tapes), as the benchmark runs it: the momentum and energy closed forms of
    test_adjoint_conservation_closed_forms hold for every particle, since every step conserves both exactly."""
    wl = W.differentiable()
    kw = dict(method=wl.method, dt=wl.dt, fE=wl.fE, seed=wl.seed, step=0)
    sp = wl.species_of_particles()
    mw = wl.m[sp] * wl.w
    v0 = np.stack([wl.vx, wl.vy, wl.vz], axis=1)

    def cot_p(vf):
        c = np.zeros_like(vf)
        c[:, 0] = mw
        return c

    vf, gv, gw, gL = _grads(mcc, wl, kw, cot_p, n_steps=50, every=10, tape=tape)
    scale = mw * np.maximum(np.abs(v0).max(1), np.abs(vf).max(1))
    want = np.zeros_like(v0)
    want[:, 0] = mw
    assert (np.abs(gv - want).max(1) / mw).max() < 1e-9
    assert (np.abs(gw - wl.m[sp] * (v0[:, 0] - vf[:, 0])) * wl.w / scale).max() < 1e-9
    assert np.abs(gL).max() < 1e-9 * np.abs(mw[:, None] * vf).sum()

    vf, gv, gw, gL = _grads(mcc, wl, kw, lambda vf: mw[:, None] * vf, n_steps=50, every=10, tape=tape)
    e0 = (v0 ** 2).sum(1)
    ef = (vf ** 2).sum(1)
    escale = mw * np.maximum(e0, ef)
    assert (np.abs(gv - mw[:, None] * v0).max(1) * np.abs(v0).max(1) / escale).max() < 1e-9
    assert (np.abs(gw - 0.5 * wl.m[sp] * (e0 - ef)) * wl.w / escale).max() < 1e-9
    assert np.abs(gL).max() < 1e-9 * (mw * ef).sum()


@pytest.mark.parametrize("case", ["even", "poisson"])
@pytest.mark.parametrize("method", [W.TA77, W.N97])
def test_adjoint_matches_oracle_finite_differences(mcc, method, case):
    """A random cotangent: sampled entries of dL/dv, dL/dw and dL/dlnL against central differences of the oracle
    step (samples whose difference quotients at h and h/2 disagree straddle a decision and are skipped)."""
    wl, kw = _case(method) if case == "even" else _poisson_case(method)
    rng = np.random.default_rng(11)
    cot = rng.standard_normal((wl.n, 3))
    vf, gv, gw, gL = _grads(mcc, wl, kw, lambda vf: cot)
    v0 = np.stack([wl.vx, wl.vy, wl.vz], axis=1)
    args = (wl.offsets, wl.n_cells, wl.n_species, wl.q, wl.m, wl.lnL, O.Params(**kw), 2)
    checked = 0
    for idx in rng.choice(wl.n, 10, replace=False):
        idx = int(idx)
        for d in range(3):
            g, g2, same = G.fd_derivative(cot, v0, wl.w, *args, ("v", idx, d))
            tol = 1e-6 * max(abs(g), np.abs(cot).max())
            if same and abs(g - g2) <= tol:
                assert abs(gv[idx, d] - g) <= tol, (idx, d, gv[idx, d], g)
                checked += 1
        seg = np.searchsorted(wl.offsets, idx, side="right") - 1
        a, b = wl.offsets[seg], wl.offsets[seg + 1]
        if np.count_nonzero(wl.w[a:b] == wl.w[idx]) > 1:
            continue  # a weight tied with another one of its population: w_max and the weight order are not smooth
        g, g2, same = G.fd_derivative(cot, v0, wl.w, *args, ("w", idx))
        tol = 1e-6 * max(abs(g), np.abs(cot).max() * np.abs(v0).max() / wl.w[idx])
        if same and abs(g - g2) <= tol:
            assert abs(gw[idx] - g) <= tol, (idx, gw[idx], g)
            checked += 1
    for a, b in ((0, 0), (0, 1), (1, 1)):
        if abs(gL[a, b]) == 0.0 and case == "poisson":
            continue
        g, g2, same = G.fd_derivative(cot, v0, wl.w, *args, ("lnL", a, b))
        tol = 1e-6 * max(abs(g), 1e-3 * np.abs(cot * v0).sum() / wl.lnL[a, b])
        if same and abs(g - g2) <= tol:
            assert abs(gL[a, b] - g) <= tol, (a, b, gL[a, b], g)
            checked += 1
    assert checked >= 25


@pytest.mark.parametrize("case", ["even", "poisson"])
@pytest.mark.parametrize("method", [W.TA77, W.N97])
def test_adjoint_equals_oracle_autodiff(mcc, method, case):
    """A random cotangent over two steps: every entry of dL/dv, dL/dw and dL/dlnL of the CUDA adjoint against the
    reverse-mode oracle gradient (torch autograd through the step transcribed on the CPU, decisions held fixed).
    Tolerance 1e-9 of each gradient's largest entry (FP64 on both sides, different summation orders)."""
    wl, kw = _case(method, n_cells=8, per_species=24) if case == "even" else _poisson_case(method)
    rng = np.random.default_rng(17)
    cot = rng.standard_normal((wl.n, 3))
    vf, gv, gw, gL = _grads(mcc, wl, kw, lambda vf: cot)
    v0 = np.stack([wl.vx, wl.vy, wl.vz], axis=1)
    vo, gvo, gwo, gLo = AD.gradient(cot, v0, wl.w, wl.lnL, wl.offsets, wl.n_cells, wl.n_species, wl.q, wl.m,
                                    O.Params(**kw), 2)
    assert np.abs(vf - vo).max() <= 1e-12 * np.abs(vo).max()
    assert np.abs(gv - gvo).max() <= 1e-9 * np.abs(gvo).max(), np.unravel_index(np.argmax(np.abs(gv - gvo)), gv.shape)
    assert np.abs(gw - gwo).max() <= 1e-9 * np.abs(gwo).max(), int(np.argmax(np.abs(gw - gwo)))
    assert np.abs(gL - gLo).max() <= 1e-9 * np.abs(gLo).max(), (gL, gLo)


@pytest.mark.parametrize("case", ["even", "poisson"])
def test_adjoint_recorded_tape(mcc, case):
    """Recorded tapes (the forward through the adjoint kernel, the backward the reverse sweep alone): the forward
    equals the oracle step, and the gradient equals the checkpointing mode's and the reverse-mode oracle gradient
    entry by entry."""
    wl, kw = _case(W.N97, n_cells=8, per_species=24) if case == "even" else _poisson_case(W.N97)
    rng = np.random.default_rng(23)
    cot = rng.standard_normal((wl.n, 3))
    vt, gvt, gwt, gLt = _grads(mcc, wl, kw, lambda vf: cot, n_steps=3, tape=True)
    vc, gvc, gwc, gLc = _grads(mcc, wl, kw, lambda vf: cot, n_steps=3, every=2)
    v0 = np.stack([wl.vx, wl.vy, wl.vz], axis=1)
    vo, gvo, gwo, gLo = AD.gradient(cot, v0, wl.w, wl.lnL, wl.offsets, wl.n_cells, wl.n_species, wl.q, wl.m,
                                    O.Params(**kw), 3)
    assert np.abs(vt - vo).max() <= 1e-12 * np.abs(vo).max()
    for a, b, c in ((gvt, gvc, gvo), (gwt, gwc, gwo), (gLt, gLc, gLo)):
        assert np.abs(a - b).max() <= 1e-9 * np.abs(c).max()
        assert np.abs(a - c).max() <= 1e-9 * np.abs(c).max()


def test_adjoint_replay_without_record_rejected(mcc):
    """A replaying call cannot also ask for the forward outputs (it runs no forward)."""
    import torch
    wl, kw = _case(W.N97)
    v, w, off, _ = _tensors(wl)
    sp = list(zip(wl.q.tolist(), wl.m.tolist()))
    mc = int(wl.counts.sum(1).max())
    buf = torch.empty(mcc.adjoint_tape_bytes(0, wl.n_cells, mc, 8), dtype=torch.uint8, device="cuda")
    out = [torch.empty_like(x) for x in v]
    with pytest.raises(mcc.MccError):
        mcc.mcc_adjoint(*v, w, off, wl.n_cells, wl.n_species, sp, wl.lnL, 0, 0, 0, mcc.Params(**kw), mc, out=out,
                        tape=mcc.ADJOINT_REPLAY, tape_buffer=buf)


def test_adjoint_checkpoint_segments_agree(mcc):
    """The backward replays each checkpoint segment: segments of 1, 3 and 10 steps give the same gradient."""
    wl, kw = _case(W.N97, n_cells=8, per_species=32)
    rng = np.random.default_rng(3)
    cot = rng.standard_normal((wl.n, 3))
    res = [_grads(mcc, wl, kw, lambda vf: cot, n_steps=4, every=e) for e in (1, 3, 10)]
    for r in res[1:]:
        assert np.allclose(r[1], res[0][1], rtol=1e-9, atol=1e-9 * np.abs(res[0][1]).max())
        assert np.allclose(r[2], res[0][2], rtol=1e-9, atol=1e-9 * np.abs(res[0][2]).max())
        assert np.allclose(r[3], res[0][3], rtol=1e-9, atol=1e-9 * np.abs(res[0][3]).max())


def test_adjoint_fp32_variant(mcc):
    """FP32 variant (mixed-precision forward, FP64 adjoint replayed from float checkpoints): the momentum closed form
    holds exactly, and the gradient of a random cotangent agrees with the FP64 variant on the same float-rounded
    inputs to float-rounding level."""
    import torch
    wl, kw = _case(W.N97, n_cells=16, per_species=64)
    for x in (wl.vx, wl.vy, wl.vz):
        x[:] = x.astype(np.float32).astype(np.float64)
    rng = np.random.default_rng(5)
    cot = rng.standard_normal((wl.n, 3))
    sp = list(zip(wl.q.tolist(), wl.m.tolist()))
    res = {}
    for dt in (torch.float64, torch.float32):
        v = [torch.tensor(x, dtype=dt, device="cuda", requires_grad=True) for x in (wl.vx, wl.vy, wl.vz)]
        w = torch.tensor(wl.w, dtype=torch.float64, device="cuda", requires_grad=True)
        L = torch.tensor(np.asarray(wl.lnL, dtype=np.float64), requires_grad=True)
        off = torch.tensor(wl.offsets, device="cuda")
        out = mcc.collision_steps(*v, w, L, off, wl.n_cells, wl.n_species, sp, mcc.Params(**kw), 2)
        c = torch.tensor(cot, device="cuda", dtype=dt)
        sum((c[:, d] * out[d]).sum() for d in range(3)).backward()
        assert v[0].grad.dtype == dt
        res[dt] = (np.stack([x.grad.double().cpu().numpy() for x in v], 1), w.grad.cpu().numpy(), L.grad.numpy())
    g64, g32 = res[torch.float64], res[torch.float32]
    for a, b in zip(g32, g64):
        assert np.abs(a - b).max() <= 1e-4 * np.abs(b).max()


def test_adjoint_rejects_unsupported_steps(mcc):
    """The adjoint covers the FP64, non-relativistic step with the paper's s and order-N pairs; anything else is an
    argument error before any launch."""
    import torch
    wl, kw = _case(W.N97)
    v, w, off, _ = _tensors(wl)
    sp = list(zip(wl.q.tolist(), wl.m.tolist()))
    mc = int(wl.counts.sum(1).max())
    out = [torch.empty_like(x) for x in v]
    for bad in ({"relativistic": True}, {"weighting": 1}, {"pairing": 1}):
        with pytest.raises(mcc.MccError) as e:
            mcc.mcc_adjoint(*v, w, off, wl.n_cells, wl.n_species, sp, wl.lnL, 0, 1, 1, mcc.Params(**kw, **bad), mc,
                            out=out)
        assert e.value.code == -1
    vf = [x.float() for x in v]
    with pytest.raises(mcc.MccError):
        mcc.mcc_adjoint(*vf, w, off, wl.n_cells, wl.n_species, sp, wl.lnL, 0, 1, 1, mcc.Params(**kw), mc, out=out)
