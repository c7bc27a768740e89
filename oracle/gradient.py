"""Oracle gradient of the collision step: central finite differences of the FP64 oracle.

TEST INFRASTRUCTURE ONLY (see the package header). The pathwise gradient the CUDA adjoint computes holds every random
draw and every discrete decision of the step fixed: the Philox draws, the permutations and pairs, the accept test of
the heavier particle, the weight order, the energy-correction pass structure and the crossing pair. Between those
decisions the step is a smooth function of the initial velocities v, the weights w and the Coulomb logarithms lnL
(Sec. 3.2 s, Eq. vp_pm, Eq. Econs, Eq. DeltaEs, Eqs. vp1/vp2/U_inelastic), so its derivative is the limit of
central differences of the oracle's own step with the same seed. This module takes that limit numerically:

    dL/dx ~ (L(x + h e) - L(x - h e)) / (2 h),   L = sum_p cot_p . v_p(after n_steps)

for a linear functional L given by a cotangent ``cot`` (N x 3). A perturbation that flips a decision makes the
difference quotient jump; ``fd_derivative`` therefore also returns the quotient at h/2 so that a caller can reject a
sample whose two estimates disagree (a decision boundary within h).

Pins (tests/test_oracle_gradient.py): exact momentum and energy conservation of every interaction fix closed-form
gradients for the cotangents m w e_x (momentum) and m w v_final (energy), for v, w and lnL.
"""
from __future__ import annotations

import numpy as np

from . import Params, State, step


def _run(vx, vy, vz, w, offsets, n_cells, S, q, m, lnL, p: Params, n_steps: int):
    st = State(vx, vy, vz, w, offsets, n_cells, S)
    corr, fail = step(st, q, m, lnL, p, n_steps=n_steps)
    return st.v(), corr, fail


def forward(v0: np.ndarray, w: np.ndarray, offsets, n_cells: int, S: int, q, m, lnL, p: Params, n_steps: int):
    """Velocities after n_steps oracle steps (a copy; inputs untouched), with the per-cell correction pairs and
    failure counts (the discrete outcome of the correction)."""
    return _run(v0[:, 0], v0[:, 1], v0[:, 2], w, offsets, n_cells, S, q, m, lnL, p, n_steps)


def loss(cot: np.ndarray, v0, w, offsets, n_cells, S, q, m, lnL, p, n_steps) -> float:
    v, _, _ = forward(v0, w, offsets, n_cells, S, q, m, lnL, p, n_steps)
    return float(np.sum(cot * v))


def fd_derivative(cot, v0, w, offsets, n_cells, S, q, m, lnL, p: Params, n_steps: int, what: tuple,
                  rel_h: float = 1e-6):
    """Central difference of L along one input: what = ("v", particle, component) | ("w", particle) |
    ("lnL", a, b) (the symmetric pair a, b). Returns (derivative at h, derivative at h/2, decisions unchanged)."""
    v0 = np.array(v0, dtype=np.float64)
    w = np.array(w, dtype=np.float64)
    L = np.array(lnL, dtype=np.float64)
    if L.ndim == 0:
        L = np.full((S, S), float(L))

    def at(delta):
        vv, ww, LL = v0.copy(), w.copy(), L.copy()
        if what[0] == "v":
            vv[what[1], what[2]] += delta
        elif what[0] == "w":
            ww[what[1]] += delta
        else:
            a, b = what[1], what[2]
            LL[a, b] += delta
            if a != b:
                LL[b, a] += delta
        vf, corr, fail = forward(vv, ww, offsets, n_cells, S, q, m, LL, p, n_steps)
        return float(np.sum(cot * vf)), corr, fail

    if what[0] == "v":
        scale = max(np.abs(v0[what[1]]).max(), 1e-300)
    elif what[0] == "w":
        scale = w[what[1]]
    else:
        scale = L[what[1], what[2]]
    h = rel_h * scale
    _, c0, f0 = at(0.0)
    lp, cp, fp = at(h)
    lm, cm, fm = at(-h)
    lp2, _, _ = at(0.5 * h)
    lm2, _, _ = at(-0.5 * h)
    same = (np.array_equal(c0, cp) and np.array_equal(c0, cm) and np.array_equal(f0, fp) and np.array_equal(f0, fm))
    return (lp - lm) / (2 * h), (lp2 - lm2) / h, same
