"""GPU parity of PIC coupling (push, multi-array gather, and the push / re-bin / collision loop) against the oracle.

The push is reproducible bit for bit (every operation rounded in the positions' precision, no fused multiply-add):
positions and cell ids must be identical. The loop compares the re-binned offsets exactly and the velocities with
the step's tolerances."""
import numpy as np
import pytest

import oracle as O
from paper_2407_19151_gb300 import workloads as W

from _parity import F32_TOL, F64_TOL, velocity_error

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mcc():
    import paper_2407_19151_gb300 as m
    m.build()
    return m


def _t(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _push_inputs(n, dtype, rel, seed):
    rng = np.random.default_rng(seed)
    grid = ((7, 5, 3), (7.0, 2.5, 4.5))
    L = grid[1]
    pos = [np.minimum((rng.random(n) * l).astype(dtype), np.nextafter(dtype(l), dtype(0))) for l in L]
    scale = 10.0 ** rng.integers(-3, 2, n)
    vel = [(rng.normal(0, 2, n) * scale).astype(dtype) for _ in range(3)]
    if n >= 8:
        # edge cases: at the walls, moves of exactly a box length, several box lengths, non-finite velocities
        pos[0][:4] = [0, np.nextafter(dtype(L[0]), dtype(0)), 0, 3]
        vel[0][:8] = [-1e-30, 1e-7, 7 / 0.6, -700.0, np.inf, -np.inf, np.nan, 0.0]
    return grid, pos, vel


@pytest.mark.parametrize("dtype", [np.float64, np.float32], ids=["f64", "f32"])
@pytest.mark.parametrize("rel", [False, True], ids=["classical", "relativistic"])
@pytest.mark.parametrize("n", [1, 1000 + 37, 300_001])
def test_push_bit_exact(mcc, dtype, rel, n):
    grid, pos, vel = _push_inputs(n, dtype, rel, seed=n + 3 * rel)
    dt = 0.6
    X = [_t(p) for p in pos]
    V = [_t(v) for v in vel]
    cell = mcc.mcc_push(*X, *V, grid, dt, relativistic=rel, c=1.0)
    ref = O.push(*pos, *vel, grid, dt, relativistic=rel, c=1.0)
    for d in range(3):
        np.testing.assert_array_equal(X[d].cpu().numpy(), ref[d])
    np.testing.assert_array_equal(cell.cpu().numpy(), ref[3])


def test_push_empty_and_invalid(mcc):
    import torch
    e = torch.empty(0, dtype=torch.float32, device="cuda")
    cell = mcc.mcc_push(e, e, e, e, e, e, ((2, 2, 2), (1.0, 1.0, 1.0)), 0.1)
    assert cell.numel() == 0
    x = torch.zeros(4, dtype=torch.float64, device="cuda")
    with pytest.raises(mcc.MccError):
        mcc.mcc_push(x, x, x, x, x, x, ((0, 2, 2), (1.0, 1.0, 1.0)), 0.1)
    with pytest.raises(mcc.MccError):
        mcc.mcc_push(x, x, x, x, x, x, ((2, 2, 2), (1.0, -1.0, 1.0)), 0.1)
    with pytest.raises(mcc.MccError):
        mcc.mcc_push(x, x, x, x, x, x, ((2, 2, 2), (1.0, 1.0, 1.0)), float("nan"))


@pytest.mark.parametrize("n", [0, 1, 5000 + 3])
def test_gather_n_exact(mcc, n):
    import torch
    rng = np.random.default_rng(n)
    perm = rng.permutation(n).astype(np.int32)
    arrs = [rng.normal(size=n), rng.normal(size=n).astype(np.float32), rng.integers(0, 9, n).astype(np.int32),
            rng.normal(size=n), rng.integers(-5, 5, n).astype(np.int64)]
    outs = mcc.mcc_gather_n([_t(a) for a in arrs], _t(perm) if n else torch.empty(0, dtype=torch.int32,
                                                                                          device="cuda"))
    for a, o in zip(arrs, outs):
        np.testing.assert_array_equal(o.cpu().numpy(), a[perm])


def _oracle_loop(wl, dtype, n_steps, cfl=0.5, order="stable", v0=None):
    """The push / bin / gather / step sequence through the oracle: positions and velocities stored in the given
    precision for the push, FP64 for the collision step."""
    grid, x, y, z, dt_push = W.pic_setup(wl, cfl=cfl)
    npdt = np.float64 if dtype == "f64" else np.float32
    sp = wl.species_of_particles()
    v = [np.asarray(a, dtype=npdt) for a in (v0 if v0 is not None else (wl.vx, wl.vy, wl.vz))]
    pos = [np.asarray(a, dtype=npdt) for a in (x, y, z)]
    w, s = wl.w.copy(), sp.copy()
    for t in range(n_steps):
        xo, yo, zo, cell = O.push(*pos, *v, grid, dt_push, relativistic=wl.relativistic, c=wl.c)
        perm, off = O.bin_particles_weighted(cell, s, w, wl.n_cells, wl.n_species) if order == "weight" else \
            O.bin_particles(cell, s, wl.n_cells, wl.n_species)
        pos = [a[perm] for a in (xo, yo, zo)]
        v = [a[perm] for a in v]
        w, s = w[perm], s[perm]
        st = O.State(*[a.astype(np.float64) for a in v], w, off, wl.n_cells, wl.n_species)
        _, rf = O.step(st, wl.q, wl.m, wl.lnL, O.Params(**dict(_base(wl), step=3 + t)), n_steps=1)
        vv = st.v()
        v = [vv[:, d].astype(npdt) for d in range(3)]
    return pos, v, w, s, off, st.v(), rf


def _base(wl):
    return dict(method=wl.method, relativistic=wl.relativistic, dt=wl.dt, dV=wl.dV, eps0=wl.eps0, c=wl.c, fE=wl.fE,
                seed=wl.seed, step=3)


def _loop_pair(mcc, wl, dtype, n_steps, cfl=0.5, order="stable"):
    """The PicLoop on the GPU and the same sequence through the oracle."""
    import torch
    grid, x, y, z, dt_push = W.pic_setup(wl, cfl=cfl)
    tdt = torch.float64 if dtype == "f64" else torch.float32
    npdt = np.float64 if dtype == "f64" else np.float32
    sp = wl.species_of_particles()
    v = [np.asarray(a, dtype=npdt) for a in (wl.vx, wl.vy, wl.vz)]
    pos = [np.asarray(a, dtype=npdt) for a in (x, y, z)]
    loop = mcc.PicLoop(*[_t(a) for a in pos], *[_t(a).to(tdt) for a in v], _t(wl.w), _t(sp), _t(wl.offsets),
                       wl.n_cells, wl.n_species, grid, list(zip(wl.q.tolist(), wl.m.tolist())), wl.lnL,
                       mcc.Params(**_base(wl)), dt_push, order=order)
    _, fail = loop.step(n_steps)
    mcc.sync_status(0)
    got = [a.cpu().numpy() for a in loop.state]
    pos, v, w, s, off, vref, rf = _oracle_loop(wl, dtype, n_steps, cfl, order)
    ok = np.repeat(fail.cpu().numpy() == rf, np.diff(off[::wl.n_species]))  # last step's cells, same failures
    return got, loop.offsets.cpu().numpy(), (pos, v, w, s, off, vref), ok


@pytest.mark.parametrize("order", ["stable", "weight"])
def test_pic_loop_fp64(mcc, order):
    """Three push / re-bin / collision steps, FP64: offsets, species and weights identical, positions and velocities
    within the FP64 tolerance (re-binned stably, or with every segment by descending weight)."""
    wl = W.three_species(n_cells=60, mean_count=90, precision="f64")
    got, off, (pos, v, w, s, roff, vref), ok = _loop_pair(mcc, wl, "f64", 3, order=order)
    np.testing.assert_array_equal(off, roff)
    np.testing.assert_array_equal(got[7], s)
    np.testing.assert_array_equal(got[6], w)
    for d in range(3):
        assert np.abs(got[d] - pos[d]).max() < 1e-12
    err = velocity_error(np.stack(got[3:6], axis=1), vref, roff)
    assert err.max() < F64_TOL, err.max()


def test_pic_loop_relativistic_fp64(mcc):
    """Two relativistic push / re-bin / collision steps, FP64. Re-binning gathers, in some cells, a few co-moving
    fast beam particles whose energy-correction pair is ill-conditioned: the oracle itself moves by ~2e-12 there when
    its inputs change by one ulp, and any difference in rounding order moves it as much. Bound, per cell: every
    particle within 1e-12, or four times the oracle's own one-ulp sensitivity in that cell (measured here), whichever
    is larger; most cells keep 1e-12."""
    wl = W.relativistic_beam(n_cells=60, count_lo=16, count_hi=200, precision="f64")
    got, off, (pos, v, w, s, roff, vref), ok = _loop_pair(mcc, wl, "f64", 2)
    np.testing.assert_array_equal(off, roff)
    np.testing.assert_array_equal(got[7], s)
    rng = np.random.default_rng(0)
    v1 = [np.asarray(a, np.float64) * (1 + rng.choice([-1.0, 1.0], wl.n) * 2.0 ** -52) for a in (wl.vx, wl.vy, wl.vz)]
    *_, off1, vref1, _ = _oracle_loop(wl, "f64", 2, v0=v1)
    np.testing.assert_array_equal(off1, roff)
    S = wl.n_species
    cell_of = np.repeat(np.arange(wl.n_cells), np.diff(roff[::S]))
    sens_p = velocity_error(vref1, vref, roff)
    sens_c = np.zeros(wl.n_cells)
    np.maximum.at(sens_c, cell_of, sens_p)
    bound = np.maximum(F64_TOL, 4 * sens_c[cell_of])
    err = velocity_error(np.stack(got[3:6], axis=1), vref, roff)
    worst = int(np.argmax(err / bound))
    assert (err < bound).all(), (err[worst], sens_c[cell_of[worst]], int(cell_of[worst]))
    assert (sens_c <= F64_TOL).mean() >= 0.8


def test_pic_loop_mixed(mcc):
    """One push / re-bin / collision step on the mixed path: the push from identical float inputs gives identical
    positions and binning; the collision step within 2e-6 for every particle."""
    wl = W.three_species(n_cells=120, mean_count=120)
    got, off, (pos, v, w, s, roff, vref), ok = _loop_pair(mcc, wl, "f32", 1)
    np.testing.assert_array_equal(off, roff)
    np.testing.assert_array_equal(got[7], s)
    for d in range(3):
        np.testing.assert_array_equal(got[d], pos[d])
    err = velocity_error(np.stack([a.astype(np.float64) for a in got[3:6]], axis=1), vref, roff)
    assert ok.all()
    assert err.max() < F32_TOL, err.max()
