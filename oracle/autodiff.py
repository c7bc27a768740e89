"""Reverse-mode gradient of the oracle's collision step: the step written a second time with PyTorch CPU scalars in
FP64, differentiated by torch.autograd.

TEST INFRASTRUCTURE ONLY (see the package header). The CUDA adjoint computes the pathwise derivative of the step:
every random draw and every discrete decision is held fixed (the Philox draws, the permutations and pairs, the
accept test of the heavier particle, the weight order, the caps and the crossing pair of the energy loop, the loop
exits, the fallback), and between those decisions the step is a smooth function of the initial velocities v, the
weights w and the Coulomb logarithms lnL. This module is an independent derivative of that function: the
arithmetic of one step (Sec. 3 scatter with Eq. sab_TA77, the TA77 / N97 angle, the rotation; Sec. 4 correction with
Eq. vp_pm, Eq. Econs, Eq. DeltaEs and the energy pairs of Eqs. vp1_inelastic / vp2_inelastic / vrel_inelastic) is
transcribed here in torch operations, each decision is taken from the values exactly as the C oracle takes it, and
autograd supplies dL/dv, dL/dw and dL/dlnL for a linear functional L = sum_p cot_p . v_p(after the steps). Only
integer work comes from the C oracle (its pair lists, permutations and Philox words); every floating-point
operation is written below. Its forward equals the C oracle's step to rounding (checked in
tests/test_oracle_autodiff.py), its gradient equals central differences of the C oracle and the closed forms that
exact momentum and energy conservation fix.

Scope: FP64, non-relativistic, the paper's s (weighting 0) and order-N pairs (pairing 0), the scope of the CUDA
adjoint. Slow (torch scalar operations): cells of tens of particles, a few steps.
"""
from __future__ import annotations

import math

import numpy as np
import torch

from . import Params, n97_A, pairs, permutation, philox4x32_10

_PERM_BITS = 20
_TAG_SCAT = 3
_TRIPLET = 1


def _f(x) -> float:
    """The value of a scalar (tensor or number), for the decisions."""
    return x.item() if torch.is_tensor(x) else float(x)


def _u23(r: int) -> float:
    """Uniform on (0, 1) from the top 23 bits of a Philox word, the oracle's mapping."""
    return ((int(r) >> 9) + 0.5) * (1.0 / 8388608.0)


def _draws(seed: int, index: int, cell: int, step: int, inter: int):
    ctr = np.array([index, cell, step & 0xFFFFFFFF, (inter << 8) | _TAG_SCAT], dtype=np.uint32)
    key = np.array([seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF], dtype=np.uint32)
    r = philox4x32_10(ctr, key)
    return [_u23(x) for x in r]


def _n97_dL(A: float) -> float:
    """dL/dA of L(A) = coth A - 1/A: 1/A^2 - 1/sinh^2 A; below A = 0.5 the derivative of its Bernoulli series
    L = sum_n 2^{2n} B_{2n} A^{2n-1} / (2n)! (the closed form cancels there)."""
    if A < 0.5:
        B = [1.0 / 6, -1.0 / 30, 1.0 / 42, -1.0 / 30, 5.0 / 66, -691.0 / 2730, 7.0 / 6, -3617.0 / 510,
             43867.0 / 798, -174611.0 / 330]
        tot, fact, pow4 = 0.0, 1.0, 1.0
        for n in range(1, len(B) + 1):
            fact *= (2 * n - 1) * (2 * n)
            pow4 *= 4.0
            tot += pow4 * B[n - 1] * (2 * n - 1) * A ** (2 * n - 2) / fact
        return tot
    e = math.exp(-2.0 * A)
    return 1.0 / (A * A) - 4.0 * e / (1.0 - e) ** 2


class _N97A(torch.autograd.Function):
    """A(s), the root of coth A - 1/A = exp(-s): the value from the oracle's root, the derivative from the implicit
    function theorem, dA/ds = -exp(-s) / L'(A)."""

    @staticmethod
    def forward(ctx, s):
        A = n97_A(_f(s))
        ctx.save_for_backward(s)
        ctx.A = A
        return torch.tensor(A, dtype=torch.float64)

    @staticmethod
    def backward(ctx, g):
        (s,) = ctx.saved_tensors
        A = ctx.A
        if A == 0.0 or math.isinf(A):
            return g * 0.0
        return g * (-math.exp(-_f(s)) / _n97_dL(A))


def _angle(method: int, s, U1: float, U4: float):
    """(sin theta, 1 - cos theta) of one pair, as the oracle samples them (Sec. 3; TA77 or N97), in torch."""
    if method == 0:  # TA77: tan(theta/2) = delta ~ N(0, s/2), Box-Muller from U1 and U4
        g = math.sqrt(-2.0 * math.log(U1)) * math.cos(2.0 * math.pi * U4)
        d = torch.sqrt(0.5 * s) * g
        if abs(_f(d)) <= 1.0:
            den = 1.0 + d * d
            return 2.0 * d / den, 2.0 * d * d / den
        t = 1.0 / d
        den = 1.0 + t * t
        return 2.0 * t / den, 2.0 / den
    A = _N97A.apply(s)
    Af = _f(A)
    zero = s * 0.0
    if Af == 0.0:
        omc, opc = zero + 2.0 * U1, zero + 2.0 * (1.0 - U1)
    elif math.isinf(Af):
        omc, opc = zero, zero + 2.0
    else:
        x = U1 * torch.expm1(-2.0 * A)
        omc = -torch.log1p(x) / A if _f(x) > -0.5 else -torch.log((1.0 - U1) + U1 * torch.exp(-2.0 * A)) / A
        opc = 2.0 - omc if _f(omc) <= 1.0 else torch.log1p((1.0 - U1) * torch.expm1(2.0 * A)) / A
    omc = torch.clamp(omc, 0.0, 2.0)
    opc = torch.clamp(opc, 0.0, 2.0)
    return torch.sqrt(omc * opc), omc


def _rotate(u, sin_t, omc, phi: float):
    """du = u' - u for u rotated through theta about a uniform azimuth phi (the Takizuka-Abe form)."""
    ux, uy, uz = u[0], u[1], u[2]
    uperp = torch.sqrt(ux * ux + uy * uy)
    umag = torch.sqrt(ux * ux + uy * uy + uz * uz)
    cp, sp = math.cos(phi), math.sin(phi)
    if _f(uperp) > 0.0:
        return torch.stack([(ux / uperp) * uz * sin_t * cp - (uy / uperp) * umag * sin_t * sp - ux * omc,
                            (uy / uperp) * uz * sin_t * cp + (ux / uperp) * umag * sin_t * sp - uy * omc,
                            -uperp * sin_t * cp - uz * omc])
    return torch.stack([umag * sin_t * cp, umag * sin_t * sp, -uz * omc])


def _scatter_cell(v, w, c, slot, a0, na, b0, nb, ma, mb, kappa, p: Params, inter: int, plist):
    """Algorithm 1's pair loop for one cell and one interaction (Sec. 3, Eq. sab_TA77), in place on the list v;
    the cell's pairs sit in the oracle's pair lists from `slot`, the cell's first particle."""
    intra = b0 == a0
    pi, pj, fl = plist
    npairs = (3 + (na - 3) // 2 if na % 2 else na // 2) if intra else (max(na, nb) if na and nb else 0)
    if intra and na < 2:
        npairs = 0
    nmin = float(na - 1) if intra else float(min(na, nb))
    mu = ma * mb / (ma + mb)
    for k in range(npairs):
        i, j = int(pi[slot + k]), int(pj[slot + k])
        vi, vj = v[i], v[j]
        wi, wj = w[i], w[j]
        heavier_i = _f(wi) > _f(wj)
        wmax, wmin = (wi, wj) if heavier_i else (wj, wi)
        U1, U2, U3, U4 = _draws(p.seed, k, c, p.step, inter)
        u = vi - vj
        u2 = (u * u).sum()
        if _f(u2) == 0.0:
            continue
        umag = torch.sqrt(u2)
        s = kappa / (mu * mu) * (wmax * nmin) / (u2 * umag)
        if int(fl[slot + k]) & _TRIPLET:
            s = s * 0.5
        sin_t, omc = _angle(p.method, s, U1, U4)
        du = _rotate(u, sin_t, omc, 2.0 * math.pi * U2)
        upd_i = upd_j = True
        if _f(wi) != _f(wj):
            heavy_moves = U3 * _f(wmax) < _f(wmin)
            if heavier_i:
                upd_i = heavy_moves
            else:
                upd_j = heavy_moves
        if upd_i:
            v[i] = vi + (mu / ma) * du
        if upd_j:
            v[j] = vj - (mu / mb) * du


def _weight_order(w, perm, s0: int):
    """The optional weight sort of Algorithm 1 as the oracle keys it: descending weight on the weight's IEEE bits
    truncated to sign, exponent and 32 mantissa bits, ties in the random order."""
    bits = np.array([_f(w[s0 + int(q)]) for q in perm], dtype=np.float64).view(np.uint64)
    keys = (~bits & ~np.uint64((1 << _PERM_BITS) - 1)) | np.arange(len(perm), dtype=np.uint64)
    order = np.sort(keys) & np.uint64((1 << _PERM_BITS) - 1)
    return [s0 + int(perm[int(r)]) for r in order]


def _pair_kecm(m1, m2, v1, v2):
    d = v1 - v2
    return 0.5 * (m1 * m2 / (m1 + m2)) * (d * d).sum()


def _energy_pair(m1, m2, v1, v2, U):
    """Eqs. vp1_inelastic / vp2_inelastic: the pair's relative velocity scaled by g = sqrt(1 - U/K)."""
    vr = v1 - v2
    K = 0.5 * (m1 * m2 / (m1 + m2)) * (vr * vr).sum()
    x = U / K
    g = torch.sqrt(1.0 - x)
    gm1 = -x / (1.0 + g)
    return v1 + (m2 / (m1 + m2)) * gm1 * vr, v2 - (m1 / (m1 + m2)) * gm1 * vr


def _correct_cell(v, w, bk, c, sides, msp, p: Params, inter: int):
    """Sec. 4 for one cell and one interaction: momentum shift (Eq. vp_pm), energy violation (Eq. Econs) and its
    partition (Eq. DeltaEs), the energy-pair loops, the fallback. Returns (energy pairs, failed)."""
    nside = len(sides)
    S = torch.zeros(3, dtype=torch.float64)
    Sw = torch.zeros((), dtype=torch.float64)
    for (s0, n), ms in zip(sides, msp):
        for t in range(s0, s0 + n):
            mp = ms * w[t]
            S = S + mp * (v[t] - bk[t])
            Sw = Sw + mp * w[t]
    B = S / Sw
    for (s0, n) in sides:
        for t in range(s0, s0 + n):
            v[t] = v[t] - B * w[t]
    dE = torch.zeros((), dtype=torch.float64)
    Es = [torch.zeros((), dtype=torch.float64) for _ in range(2)]
    wsum = [torch.zeros((), dtype=torch.float64) for _ in range(2)]
    for side, ((s0, n), ms) in enumerate(zip(sides, msp)):
        for t in range(s0, s0 + n):
            mp = ms * w[t]
            dE = dE + 0.5 * mp * ((v[t] - bk[t]) * (v[t] + bk[t])).sum()
            Es[side] = Es[side] + 0.5 * mp * (v[t] * v[t]).sum()
            wsum[side] = wsum[side] + w[t]
    ns = [n for _, n in sides] + [0] * (2 - nside)
    D = [dE, torch.zeros((), dtype=torch.float64)]
    fail = False
    if nside == 2:
        can = [ns[0] >= 2, ns[1] >= 2]
        if can[0] and can[1]:
            wa = wsum[0] / float(ns[0]) * Es[0]
            wb = wsum[1] / float(ns[1]) * Es[1]
            den = wa + wb
            if _f(den) > 0.0:
                D = [wa / den * dE, None]
                D[1] = dE - D[0]
            elif _f(dE) != 0.0:
                fail = True
        elif can[0]:
            D = [dE, dE * 0.0]
        elif can[1]:
            D = [dE * 0.0, dE]
        elif _f(dE) != 0.0:
            fail = True
    # "Delta E_s = 0" read as: no larger than 2^-47 of the species' post-shift energy (rounding noise). The value is
    # then zero (no pairs, as in the C oracle), and the derivative is that of the limit: the first pair of the order
    # as the crossing pair with U = Delta E_s (its value 0, its derivative that of Delta E_s).
    zeroed = [abs(_f(D[side])) <= 2.0 ** -47 * _f(Es[side]) for side in range(nside)]
    used = 0
    for side in range(nside):
        if fail:
            break
        Dv = D[side] - D[side].detach() if zeroed[side] else D[side]
        s0, n = sides[side]
        if zeroed[side] or _f(Dv) == 0.0:
            if n >= 2 and torch.is_tensor(Dv) and Dv.requires_grad:
                perm = permutation(n, p.seed, p.step, c, inter, side)
                rho = _weight_order(w, perm, s0) if p.sort_by_weight else [s0 + int(q) for q in perm]
                i, j = rho[0], rho[1]
                m1, m2 = msp[side] * w[i], msp[side] * w[j]
                if _f(_pair_kecm(m1, m2, v[i], v[j])) > 0.0:
                    v[i], v[j] = _energy_pair(m1, m2, v[i], v[j], Dv)
            continue
        perm = permutation(n, p.seed, p.step, c, inter, side)
        rho = _weight_order(w, perm, s0) if p.sort_by_weight else [s0 + int(q) for q in perm]
        for pas in range(p.max_corr_passes):
            if _f(Dv) == 0.0:
                break
            t = pas % 2
            while t + 1 < n and _f(Dv) != 0.0:
                i, j = rho[t], rho[t + 1]
                m1, m2 = msp[side] * w[i], msp[side] * w[j]
                K = _pair_kecm(m1, m2, v[i], v[j])
                if _f(K) > 0.0:
                    capE = p.fE * K
                    U = capE if abs(_f(Dv)) >= _f(capE) else torch.abs(Dv)
                    U = U if _f(Dv) > 0.0 else -U
                    v[i], v[j] = _energy_pair(m1, m2, v[i], v[j], U)
                    Dv = Dv - U
                    used += 1
                t += 2
        if _f(Dv) != 0.0:
            fail = True
    if fail and p.fail_policy == 0:
        for (s0, n) in sides:
            for t in range(s0, s0 + n):
                v[t] = bk[t]
    return used, fail


def step(v0, w, lnL, offsets, n_cells: int, n_species: int, q, m, p: Params, n_steps: int = 1, interactions=None):
    """n_steps collision steps of the state (v0: (N, 3) tensor, w: (N,) tensor, lnL: (S, S) tensor, FP64, any of
    them requiring grad). Returns the (N, 3) velocities after the steps as a differentiable tensor."""
    if p.relativistic or p.weighting != 0 or p.pairing != 0:
        raise ValueError("the autodiff oracle covers the non-relativistic step with the paper's s and order-N pairs")
    offsets = np.asarray(offsets, dtype=np.int64)
    S = n_species
    inters = [(a, b) for a in range(S) for b in range(a, S)] if interactions is None else \
        [tuple(int(x) for x in ab) for ab in interactions]
    v = list(v0.unbind(0))
    wl = list(w.unbind(0))
    q = [float(x) for x in q]
    m = [float(x) for x in m]
    base_step = int(p.step)
    for t in range(n_steps):
        pt = Params(**{**p.__dict__, "step": base_step + t})
        for k, (a, b) in enumerate(inters):
            plist = pairs(offsets, n_cells, S, a, b, k, pt.seed, pt.step)
            kappa = q[a] * q[a] * q[b] * q[b] * lnL[a, b] * pt.dt / (4.0 * math.pi * pt.eps0 * pt.eps0 * pt.dV)
            for c in range(n_cells):
                a0, na = int(offsets[c * S + a]), int(offsets[c * S + a + 1] - offsets[c * S + a])
                b0, nb = int(offsets[c * S + b]), int(offsets[c * S + b + 1] - offsets[c * S + b])
                intra = a == b
                if (na < 2) if intra else (na == 0 or nb == 0):
                    continue
                sides = [(a0, na)] if intra else [(a0, na), (b0, nb)]
                bk = {}
                for s0, n in sides:
                    for i in range(s0, s0 + n):
                        bk[i] = v[i]
                _scatter_cell(v, wl, c, int(offsets[c * S]), a0, na, b0, nb, m[a], m[b], kappa, pt, k, plist)
                if pt.correct:
                    _correct_cell(v, wl, bk, c, sides, [m[a]] if intra else [m[a], m[b]], pt, k)
    return torch.stack(v)


def gradient(cot, v0, w, lnL, offsets, n_cells: int, n_species: int, q, m, p: Params, n_steps: int = 1):
    """(velocities after the steps, dL/dv0 (N, 3), dL/dw (N,), dL/dlnL (S, S)) for L = sum cot * v(after), all
    numpy FP64. dL/dlnL[a, b] (a <= b) is the derivative with respect to the logarithm of interaction (a, b)."""
    V = torch.tensor(np.asarray(v0, dtype=np.float64), requires_grad=True)
    W = torch.tensor(np.asarray(w, dtype=np.float64), requires_grad=True)
    L = np.asarray(lnL, dtype=np.float64)
    L = torch.tensor(np.full((n_species, n_species), float(L)) if L.ndim == 0 else L, requires_grad=True)
    out = step(V, W, L, offsets, n_cells, n_species, q, m, p, n_steps)
    (torch.tensor(np.asarray(cot, dtype=np.float64)) * out).sum().backward()
    return out.detach().numpy(), V.grad.numpy(), W.grad.numpy(), L.grad.numpy()
