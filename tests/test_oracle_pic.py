"""Pins of the oracle's PIC-coupling push (free streaming of Eq. Boltzmann's left-hand side with a = 0, periodic box)
against exact arithmetic: dyadic cases that no rounding touches, cell ids against exact rational floors, wrapped
positions against exact rational remainders, relativistic displacements against 50-digit decimal arithmetic, and
the global moments of a push / re-bin / collision step."""
from decimal import Decimal, getcontext
from fractions import Fraction

import numpy as np
import pytest

import oracle as O
from paper_2407_19151_gb300 import workloads as W

BOX = ((4, 2, 3), (4.0, 1.0, 6.0))   # cell widths 1, 0.5, 2


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_dyadic_moves_and_wraps(dtype):
    # (x, v, dt) -> x' exactly, on the first axis (L = 4, unit cells)
    cases = [(1.25, 0.5, 0.25, 1.375), (3.75, 1.0, 0.5, 0.25), (0.25, -1.0, 0.5, 3.75), (1.0, 21.0, 2.0, 3.0),
             (2.0, -10.0, 1.0, 0.0), (0.0, 0.0, 1.0, 0.0), (3.5, 0.25, 2.0, 0.0)]
    x = np.array([c[0] for c in cases], dtype)
    v = np.array([c[1] for c in cases], dtype)
    dt = 0.25
    # scale the per-case dt into the velocity so that one dt serves all cases (all values stay dyadic)
    v = (v * np.array([c[2] for c in cases], dtype) / dtype(dt)).astype(dtype)
    zero = np.zeros_like(x)
    half = np.full_like(x, 0.25)
    nx, ny, nz = BOX[0]
    xo, yo, zo, cell = O.push(x, half, np.ones_like(x), v, zero, zero, BOX, dt)
    np.testing.assert_array_equal(xo, np.array([c[3] for c in cases], dtype))
    np.testing.assert_array_equal(yo, half)
    ix = np.floor(np.array([c[3] for c in cases])).astype(np.int32)
    np.testing.assert_array_equal(cell, ix + nx * (0 + ny * 0))


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_positions_are_exact_remainders_and_cells_exact_floors(dtype):
    rng = np.random.default_rng(3)
    n = 3000
    (nx, ny, nz), (lx, ly, lz) = BOX
    L = [lx, ly, lz]
    pos = [(rng.random(n) * l).astype(dtype) for l in L]
    pos = [np.minimum(p, np.nextafter(dtype(l), dtype(0))) for p, l in zip(pos, L)]
    vel = [(rng.normal(0, 3, n) * (10.0 ** rng.integers(-3, 2, n))).astype(dtype) for _ in range(3)]
    dt = 0.37
    out = O.push(*pos, *vel, BOX, dt)
    eps = float(np.finfo(dtype).eps)
    tdt = Fraction(float(dtype(dt)))
    for d in range(3):
        Ld = Fraction(float(dtype(L[d])))
        for i in range(0, n, 7):
            xn = Fraction(float(out[d][i]))
            assert 0 <= xn < Ld
            # the exact periodic image of x + v dt, within the rounding of the product and sum (a few ulps of the
            # larger of |x + v dt| and L)
            exact = Fraction(float(pos[d][i])) + Fraction(float(vel[d][i])) * tdt
            image = exact - (exact // Ld) * Ld
            dist = min(abs(xn - image), Ld - abs(xn - image))
            scale = max(abs(float(exact)), float(Ld))
            assert float(dist) <= 4 * eps * scale, (d, i, float(dist))
    # the cell id is the exact floor of x' nx / L except within a rounding of a cell boundary
    sx = [dtype(nx / lx), dtype(ny / ly), dtype(nz / lz)]
    ncs = (nx, ny, nz)
    for i in range(n):
        ids = []
        for d in range(3):
            t = Fraction(float(out[d][i])) * Fraction(float(sx[d]))
            k = min(int(t), ncs[d] - 1)
            frac = float(t - int(t))
            near = frac < 4 * eps * max(1.0, float(t)) or 1 - frac < 4 * eps * max(1.0, float(t))
            got = (int(out[3][i]) // (1, nx, nx * ny)[d]) % ncs[d]
            assert got == k or near, (i, d, got, k)
            ids.append(got)
        assert int(out[3][i]) == ids[0] + nx * (ids[1] + ny * ids[2])


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_relativistic_displacement(dtype):
    getcontext().prec = 50
    rng = np.random.default_rng(5)
    n = 400
    c = 1.0
    u = [(rng.normal(0, 1, n) * 10.0 ** rng.uniform(-2, 1, n)).astype(dtype) for _ in range(3)]
    big = ((1000,) * 3, (1000.0,) * 3)
    x0 = [np.full(n, 500.0, dtype) for _ in range(3)]
    dt = 0.75
    out = O.push(*x0, *u, big, dt, relativistic=True, c=c)
    eps = float(np.finfo(dtype).eps)
    for i in range(n):
        uu = [Decimal(float(u[d][i])) for d in range(3)]
        gam = (1 + sum(q * q for q in uu) / Decimal(c) ** 2).sqrt()
        speed2 = Decimal(0)
        for d in range(3):
            want = uu[d] / gam * Decimal(float(dtype(dt)))
            got = Decimal(float(out[d][i])) - Decimal(500)
            # rounding of gamma, of the velocity, of the step and of the sum at x ~ 500
            tol = Decimal(8 * eps) * abs(want) + Decimal(eps * 500)
            assert abs(got - want) <= tol, (i, d, float(got), float(want))
            speed2 += (uu[d] / gam) ** 2
        assert speed2 < Decimal(c) ** 2


def test_non_finite_and_edge_positions():
    L = 4.0
    for dtype in (np.float64, np.float32):
        tiny = np.finfo(dtype).tiny
        x = np.array([0.0, 0.0, 3.0, 1.0], dtype)
        v = np.array([-tiny, np.inf, np.nan, -4.0], dtype)
        o = O.push(x, x, x, v, v, v, ((4, 4, 4), (L, L, L)), 1.0)
        assert np.all((o[0] >= 0) & (o[0] < L))
        assert o[0][1] == 0 and o[0][2] == 0          # non-finite positions become 0
        assert o[0][3] == 1.0                          # a move of exactly -L returns to the start
        assert np.all((o[3] >= 0) & (o[3] < 64))


def test_push_rebin_collide_conserves_global_moments():
    """One PIC step (push, cell sort, gather, collision step) conserves the total momentum and energy: the push
    moves no velocity and every cell's collision step conserves both exactly."""
    wl = W.three_species(n_cells=24, mean_count=60, precision="f64")
    grid, x, y, z, dt_push = W.pic_setup(wl, cfl=0.5)
    sp = wl.species_of_particles()
    m = wl.m[sp] * wl.w
    P0 = np.array([np.sum(m * v) for v in (wl.vx, wl.vy, wl.vz)])
    E0 = 0.5 * np.sum(m * (wl.vx ** 2 + wl.vy ** 2 + wl.vz ** 2))
    xo, yo, zo, cell = O.push(x, y, z, wl.vx, wl.vy, wl.vz, grid, dt_push)
    moved = np.mean(cell != wl.cell_of_particles())
    assert 0.05 < moved < 0.9
    perm, off = O.bin_particles(cell, sp, wl.n_cells, wl.n_species)
    assert np.all(np.diff(cell[perm].astype(np.int64) * wl.n_species + sp[perm]) >= 0)
    st = O.State(wl.vx[perm], wl.vy[perm], wl.vz[perm], wl.w[perm], off, wl.n_cells, wl.n_species)
    p = O.Params(method=wl.method, dt=wl.dt, dV=wl.dV, eps0=wl.eps0, c=wl.c, fE=wl.fE, seed=wl.seed)
    O.step(st, wl.q, wl.m, wl.lnL, p, n_steps=1)
    v = st.v()
    m1 = wl.m[sp[perm]] * wl.w[perm]
    P1 = np.array([np.sum(m1 * v[:, d]) for d in range(3)])
    E1 = 0.5 * np.sum(m1 * (v ** 2).sum(1))
    scale = np.sum(m * np.sqrt(wl.vx ** 2 + wl.vy ** 2 + wl.vz ** 2))
    assert np.abs(P1 - P0).max() < 1e-12 * scale
    assert abs(E1 - E0) < 1e-12 * E0
