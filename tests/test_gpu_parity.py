"""GPU parity: every C-ABI call against the FP64 oracle on the same seeded inputs.

Bar (spec tolerances): binning and pairing bit-exact; FP64 velocities within 1e-12 of the oracle (relative to
the population's rms speed); energy-pair counts and failure flags equal. The mixed path (float velocities, float
pair kinematics) within 2e-6 for every particle, with the same failure flags.
"""
import numpy as np
import pytest

import oracle as O
from paper_2407_19151_gb300 import workloads as W

from _parity import (F32_TOL, F64_TOL, cell_moments, device_state, gpu_velocities, oracle_state,
                     velocity_error)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mcc():
    import paper_2407_19151_gb300 as m
    m.build()
    return m


def _species(wl):
    return list(zip(wl.q.tolist(), wl.m.tolist()))


def _params(mcc, wl, **kw):
    base = dict(method=wl.method, relativistic=wl.relativistic, dt=wl.dt, dV=wl.dV, eps0=wl.eps0, c=wl.c, fE=wl.fE,
                seed=wl.seed, step=7)
    base.update(kw)
    return mcc.Params(**base), O.Params(**base)


# ------------------------------------------------------------------------------------------------- binning
# segment sizes: ~50, ~24 and ~6 (one warp per segment; the last over 13 scan tiles), ~625 (one CTA, shared memory),
# ~30000 (one CTA, in place); ~171 at full size
BIN_CASES = [(0, 4, 2), (1, 1, 1), (1000, 7, 3), (200_000, 4096, 2), (300_000, 25_000, 2), (20_000, 16, 2),
             (30_000, 3, 1),
             (134_296_981, 1 << 18, 3)]  # the benchmark's full size: 1.34e8 particles in 2^18 cells x 3 species


@pytest.mark.parametrize("n,C,S", BIN_CASES)
def test_bin_bit_exact(mcc, n, C, S):
    import torch
    rng = np.random.default_rng(n + C)
    if n == 30_000:  # one huge segment: exercises the in-place (global memory) segment sort
        cell = np.zeros(n, np.int32)
        cell[::1000] = 2
    else:
        cell = rng.integers(0, C, n).astype(np.int32)
    sp = rng.integers(0, S, n).astype(np.int32)
    perm, off = mcc.mcc_bin(torch.from_numpy(cell).cuda(), torch.from_numpy(sp).cuda(), C, S)
    mcc.sync_status(0)
    rperm, roff = O.bin_particles(cell, sp, C, S)
    np.testing.assert_array_equal(off.cpu().numpy(), roff)
    np.testing.assert_array_equal(perm.cpu().numpy(), rperm)


@pytest.mark.parametrize("n,C,S", BIN_CASES)
def test_bin_weighted_bit_exact(mcc, n, C, S):
    """Weight-ordered segments: exact ties, ties below the key width, distinct weights just above it; one case
    holds a segment of ~30k particles (keys sorted in the workspace instead of shared memory)."""
    import torch
    rng = np.random.default_rng(n + C + 1)
    if n == 30_000:
        cell = np.zeros(n, np.int32)
        cell[::1000] = 2
    else:
        cell = rng.integers(0, C, n).astype(np.int32)
    sp = rng.integers(0, S, n).astype(np.int32)
    base = 10.0 ** rng.uniform(0, 4, n)
    ref = base[rng.integers(0, max(n, 1), n)] if n else base
    pick = rng.integers(0, 4, n)
    w = np.where(pick == 0, ref, np.where(pick == 1, ref * (1 + 2.0 ** -40),
                                          np.where(pick == 2, ref * (1 + 2.0 ** -30), base)))
    perm, off = mcc.mcc_bin_weighted(torch.from_numpy(cell).cuda(), torch.from_numpy(sp).cuda(),
                                     torch.from_numpy(np.ascontiguousarray(w)).cuda(), C, S)
    mcc.sync_status(0)
    rperm, roff = O.bin_particles_weighted(cell, sp, w, C, S)
    np.testing.assert_array_equal(off.cpu().numpy(), roff)
    np.testing.assert_array_equal(perm.cpu().numpy(), rperm)


def test_bin_out_of_range_latches_bounds(mcc):
    import torch
    cell = torch.tensor([0, 1, 9], dtype=torch.int32, device="cuda")
    sp = torch.zeros(3, dtype=torch.int32, device="cuda")
    mcc.mcc_bin(cell, sp, 2, 1)
    with pytest.raises(mcc.MccError) as e:
        mcc.sync_status(0)
    assert e.value.code == -6


def test_gather(mcc):
    import torch
    x = torch.arange(1000, dtype=torch.float64, device="cuda") * 0.5
    perm = torch.randperm(1000, device="cuda").to(torch.int32)
    np.testing.assert_array_equal(mcc.mcc_gather(x, perm).cpu().numpy(), x.cpu().numpy()[perm.cpu().numpy()])


# ------------------------------------------------------------------------------------------------- pairing
def _pair_cases():
    counts = np.array([[0, 0], [1, 0], [0, 1], [1, 1], [2, 0], [3, 1], [4, 7], [5, 5], [9, 2], [2, 9], [33, 1],
                       [64, 65], [257, 300], [1, 40]])
    yield "edges", counts
    yield "poisson", np.random.default_rng(3).poisson(40, size=(300, 2))


@pytest.mark.parametrize("name,counts", list(_pair_cases()))
def test_pair_bit_exact(mcc, name, counts):
    import torch
    C_, S = counts.shape
    off = np.concatenate([[0], np.cumsum(counts.reshape(-1))]).astype(np.int64)
    toff = torch.from_numpy(off).cuda()
    for k, (a, b) in enumerate([(0, 0), (0, 1), (1, 1)]):
        pi, pj, fl = mcc.mcc_pair(toff, C_, S, a, b, k, 0xABCDEF0123, 11)
        mcc.sync_status(0)
        ri, rj, rf = O.pairs(off, C_, S, a, b, k, 0xABCDEF0123, 11)
        for c in range(C_):
            na, nb = counts[c, a], counts[c, b]
            if a == b:
                npairs = 0 if na < 2 else (na // 2 if na % 2 == 0 else (na + 3) // 2)
            else:
                npairs = max(na, nb) if na and nb else 0
            s = off[c * S]
            sl = slice(s, s + npairs)
            np.testing.assert_array_equal(pi[sl].cpu().numpy(), ri[sl])
            np.testing.assert_array_equal(pj[sl].cpu().numpy(), rj[sl])
            np.testing.assert_array_equal(fl[sl].cpu().numpy(), rf[sl])


def test_pair_bit_exact_full_size(mcc):
    """The benchmark's cell counts at full size (2^18 cells x 3 species, 1.34e8 particles): the random permutations
    and the Takizuka-Abe pairs of an intra-species and two inter-species interactions, every pair slot of every cell
    bit-exact against the oracle."""
    import torch
    counts = W.three_species_counts()
    C_, S = counts.shape
    off = np.concatenate([[0], np.cumsum(counts.reshape(-1))]).astype(np.int64)
    toff = torch.from_numpy(off).cuda()
    for k, (a, b) in enumerate([(0, 0), (0, 1), (1, 2)]):
        pi, pj, fl = mcc.mcc_pair(toff, C_, S, a, b, k, 0xABCDEF0123, 11)
        mcc.sync_status(0)
        ri, rj, rf = O.pairs(off, C_, S, a, b, k, 0xABCDEF0123, 11)
        na, nb = counts[:, a], counts[:, b]
        if a == b:
            npairs = np.where(na < 2, 0, np.where(na % 2 == 0, na // 2, (na + 3) // 2))
        else:
            npairs = np.where((na > 0) & (nb > 0), np.maximum(na, nb), 0)
        # pair slot q of cell c sits at off[c S] + q
        start = off[:-1:S]
        slot = np.repeat(start, npairs) + (np.arange(npairs.sum()) - np.repeat(np.cumsum(npairs) - npairs, npairs))
        np.testing.assert_array_equal(pi.cpu().numpy()[slot], ri[slot])
        np.testing.assert_array_equal(pj.cpu().numpy()[slot], rj[slot])
        np.testing.assert_array_equal(fl.cpu().numpy()[slot], rf[slot])


# ------------------------------------------------------------------------------------------------- unfused calls
@pytest.mark.parametrize("method", [W.TA77, W.N97])
def test_scatter_then_correct_fp64(mcc, method):
    wl = W.three_species(n_cells=24, mean_count=60, precision="f64", method=method)
    v, w, off = device_state(wl, "f64")
    st = oracle_state(wl, "f64")
    pp, op = _params(mcc, wl, dt=wl.dt * 3)
    species = _species(wl)
    for k, (a, b) in enumerate(wl.interactions()):
        a, b = int(a), int(b)
        pairs = mcc.mcc_pair(off, wl.n_cells, wl.n_species, a, b, k, pp.seed, pp.step)
        backup = mcc.mcc_scatter(*v, w, off, wl.n_cells, wl.n_species, species, wl.lnL, a, b, k, pairs, pp)
        mcc.sync_status(0)
        rbk = O.scatter(st, wl.q, wl.m, wl.lnL, a, b, k, op)
        got = gpu_velocities(v)
        assert velocity_error(got, st.v(), wl.offsets).max() < F64_TOL, f"scatter {a}{b}"
        # the pre-scatter copy of the participants equals the oracle's (bit-exact before the first correction)
        sp_of = wl.species_of_particles()
        part = (sp_of == a) | (sp_of == b)
        bk = backup.cpu().numpy()[:, part]
        if k == 0:
            np.testing.assert_array_equal(bk, rbk[:, part])
        scale = np.sqrt((rbk[:, part] ** 2).sum(0)).mean()
        assert np.abs(bk - rbk[:, part]).max() / scale < F64_TOL
        corr, fail = mcc.mcc_correct(*v, w, off, wl.n_cells, wl.n_species, species, a, b, k, pp, backup)
        mcc.sync_status(0)
        rc, rf = O.correct(st, wl.m, a, b, k, op, rbk)
        got = gpu_velocities(v)
        assert velocity_error(got, st.v(), wl.offsets).max() < F64_TOL, f"correct {a}{b}"
        np.testing.assert_array_equal(corr.cpu().numpy(), rc)
        np.testing.assert_array_equal(fail.cpu().numpy(), rf)


# ------------------------------------------------------------------------------------------------- fused step
FUSED_F64 = [
    ("isotropisation", lambda: W.isotropisation(n_cells=16, per_cell=96), {}),
    ("equilibration_ta77", lambda: W.equilibration(n_cells=48, mean_count=40, precision="f64", method=W.TA77),
     {"dt_scale": 5}),
    ("equilibration_nosort", lambda: W.equilibration(n_cells=48, mean_count=40, precision="f64"),
     {"sort_by_weight": False, "dt_scale": 5}),
    ("three_species", lambda: W.three_species(n_cells=64, mean_count=90, precision="f64"), {}),
    ("differentiable", lambda: W.differentiable(n_cells=8, per_species=256), {}),
    ("momentum_only", lambda: W.relativistic_beam(n_cells=40, count_lo=4, count_hi=40, precision="f64"),
     {"fail_policy": 1, "dt_scale": 20}),
    ("relativistic", lambda: W.relativistic_beam(n_cells=40, count_lo=16, count_hi=300, precision="f64"), {}),
    ("tied_weights", lambda: _tied(W.three_species(n_cells=40, mean_count=200, precision="f64")), {}),
    ("large_segments", lambda: W.differentiable(n_cells=4, per_species=1500), {}),
    ("weight_ordered", lambda: W.three_species(n_cells=64, mean_count=90, precision="f64").weight_ordered(), {}),
    ("duplicity_weighting", lambda: W.three_species(n_cells=64, mean_count=90, precision="f64"), {"weighting": 1}),
    ("nxn_single_species", lambda: W.isotropisation(n_cells=16, per_cell=33), {"pairing": 1}),
    ("nxn_two_species", lambda: W.equilibration(n_cells=64, mean_count=16, precision="f64"), {"pairing": 1}),
    ("nxn_three_species", lambda: W.three_species(n_cells=24, mean_count=90, precision="f64"), {"pairing": 1}),
    ("duplicity_ta77", lambda: W.equilibration(n_cells=48, mean_count=40, precision="f64", method=W.TA77),
     {"weighting": 1, "dt_scale": 5}),
    ("ordered_key_ties", lambda: _key_ties(W.three_species(n_cells=40, mean_count=200, precision="f64")), {}),
    # full sizes: the isotropisation workload (64 cells x 128) and the differentiable workload's forward step
    # (1024 cells x 512, two species)
    ("isotropisation_full_size", lambda: W.isotropisation(), {}),
    ("differentiable_full_size", lambda: W.differentiable(), {}),
]


def _key_ties(wl):
    """Weight-ordered segments whose weights fall strictly but only below the sort key's 2^-32 tie width: the
    stored order is not the weight order (ties keep the random order), so the kernel must sort."""
    off = wl.offsets
    for k in range(len(off) - 1):
        n = int(off[k + 1] - off[k])
        wl.w[off[k]:off[k + 1]] = 3.0 * (1.0 + 2.0 ** -40 * np.arange(n, 0, -1))
    return wl


def _tied(wl):
    """Weights from a three-value set: ties inside every species exercise the per-interaction weight sort."""
    wl.w[:] = np.random.default_rng(5).choice([1.0, 2.0, 40.0], size=wl.n)
    return wl


def _run_fused(mcc, wl, dtype, n_steps=2, **kw):
    dt_scale = kw.pop("dt_scale", 1)
    v, w, off = device_state(wl, dtype)
    st = oracle_state(wl, dtype)
    pp, op = _params(mcc, wl, dt=wl.dt * dt_scale, **kw)
    corr, fail = mcc.mcc_step_fused(*v, w, off, wl.n_cells, wl.n_species, _species(wl), wl.lnL, pp, n_steps=n_steps)
    mcc.sync_status(0)
    rc, rf = O.step(st, wl.q, wl.m, wl.lnL, op, n_steps=n_steps)
    return gpu_velocities(v), st.v(), corr.cpu().numpy(), fail.cpu().numpy(), rc, rf


@pytest.mark.parametrize("name,make,kw", FUSED_F64, ids=[c[0] for c in FUSED_F64])
def test_fused_fp64(mcc, name, make, kw):
    wl = make()
    got, ref, corr, fail, rc, rf = _run_fused(mcc, wl, "f64", **dict(kw))
    err = velocity_error(got, ref, wl.offsets)
    assert err.max() < F64_TOL, err.max()
    np.testing.assert_array_equal(corr, rc)
    np.testing.assert_array_equal(fail, rf)


# Mixed-path cases: the group size classes at the sizes the benchmark runs (cells of ~900 particles span classes 0-3;
# a cell of 4733 particles, the benchmark's largest, class 4) and the relativistic beam with counts up to 2048.
FUSED_F32 = [
    ("equilibration_n97", lambda: W.equilibration(n_cells=200, mean_count=60, precision="f32", method=W.N97)),
    ("equilibration_ta77", lambda: W.equilibration(n_cells=200, mean_count=60, precision="f32", method=W.TA77)),
    ("three_species", lambda: W.three_species(n_cells=200, mean_count=120)),
    ("three_species_ta77", lambda: W.three_species(n_cells=200, mean_count=120, method=W.TA77)),
    ("three_species_ordered", lambda: W.three_species(n_cells=200, mean_count=120).weight_ordered()),
    ("three_species_classes", lambda: W.three_species(n_cells=64, mean_count=900)),
    ("three_species_classes_ordered", lambda: W.three_species(n_cells=64, mean_count=900).weight_ordered()),
    ("three_species_largest_cell", lambda: W.three_species(n_cells=2, mean_count=4733, sigma=0.002)),
    ("relativistic", lambda: W.relativistic_beam(n_cells=100, count_lo=16, count_hi=400)),
    ("relativistic_counts_2048", lambda: W.relativistic_beam(n_cells=24, count_lo=1500, count_hi=2048)),
]


@pytest.mark.parametrize("name,make", FUSED_F32, ids=[c[0] for c in FUSED_F32])
def test_fused_mixed_precision_scatter(mcc, name, make):
    """Mixed path, scatter phase of every interaction (correction off): every particle within 2e-6 of the FP64
    oracle run on the same float-rounded inputs."""
    wl = make()
    got, ref, corr, fail, rc, rf = _run_fused(mcc, wl, "f32", n_steps=1, correct=False)
    err = velocity_error(got, ref, wl.offsets)
    assert err.max() < F32_TOL, err.max()


@pytest.mark.parametrize("name,make", FUSED_F32, ids=[c[0] for c in FUSED_F32])
def test_fused_mixed_precision(mcc, name, make):
    """Mixed path, whole step, against the FP64 oracle run on the same float-rounded inputs: the same failed
    corrections and energy-pair counts; 99.9% of particles within 2e-6 and every particle within 1e-5. The velocities
    stay float-float on chip for the whole step and every sum, coefficient and energy pair is float-float, so the
    only difference left is the float pair kinematics (the scatter alone holds 2e-6 for every particle). It reaches
    the energy correction through Delta E_s: a large-angle scatter of heavy, heavily weighted particles exchanges
    energy with ~1e-7 relative float error, and the crossing pair of the energy loop takes the remainder of
    Delta E_s, so its two particles move by that error over the pair's CM energy (measured: 2.7e-6 for one pair of
    a C6+ cell whose remainder is 5e-4 of Delta E_s)."""
    wl = make()
    got, ref, corr, fail, rc, rf = _run_fused(mcc, wl, "f32", n_steps=1)
    err = velocity_error(got, ref, wl.offsets)
    np.testing.assert_array_equal(fail, rf)
    assert np.quantile(err, 0.999) < F32_TOL, np.quantile(err, 0.999)
    assert err.max() < 1e-5, err.max()


@pytest.mark.parametrize("name,make", [
    ("three_species", lambda: W.three_species(n_cells=1 << 18).weight_ordered()),
    ("equilibration_ta77", lambda: W.equilibration(precision="f32", method=W.TA77)),
    ("relativistic_beam", lambda: W.relativistic_beam()),
], ids=["three_species", "equilibration_ta77", "relativistic_beam"])
def test_fused_mixed_precision_full_size_sampled(mcc, name, make):
    """The mixed-precision workloads at their full sizes (three species: 2^18 cells, 1.34e8 particles, segments in
    weight order, the benchmark's workload; two-species equilibration: 4096 cells; relativistic beam: 65536 cells,
    1.16e7 particles) in the launch configuration the benchmark times (automatic class capacities, every size class,
    one fused step), checked on sampled cells against the oracle stepped on those cells alone (every draw is keyed by
    the global cell id, so a cell's step does not depend on the others): the first 512 cells, the largest cell, and
    256 cells drawn at random. The bounds of test_fused_mixed_precision: the same failed corrections, 99.9% of the
    sampled particles within 2e-6 and every one within 1e-5."""
    wl = make()
    C, S = wl.n_cells, wl.n_species
    tot = wl.counts.sum(axis=1)
    v, w, off = device_state(wl, "f32")
    pp, op = _params(mcc, wl)
    _, fail = mcc.mcc_step_fused(*v, w, off, C, S, _species(wl), wl.lnL, pp, n_steps=1, max_cell=int(tot.max()))
    mcc.sync_status(0)
    got = gpu_velocities(v)
    fail = fail.cpu().numpy()
    del v, w, off
    rng = np.random.default_rng(20240719)
    cells = np.unique(np.concatenate([np.arange(min(512, C)), [int(np.argmax(tot))],
                                      rng.choice(C, 256, replace=False)]))
    st = oracle_state(wl, "f32")
    rf = np.zeros(C, dtype=np.int32)
    for c in cells:  # one oracle call per sampled cell (its global id, its own draws)
        _, f = O.step(st, wl.q, wl.m, wl.lnL, op, n_steps=1, cell_begin=int(c), cell_end=int(c) + 1)
        rf[c] = f[c]
    np.testing.assert_array_equal(fail[cells], rf[cells])
    # the sampled cells' particles, in cell order, with their (cell, species) segment offsets among them
    sel = np.flatnonzero(np.isin(np.repeat(np.arange(C), tot), cells))
    seg = np.concatenate([[0], np.cumsum(wl.counts[cells].reshape(-1))])
    ref = np.stack([st.vx[sel], st.vy[sel], st.vz[sel]], axis=1)
    err = velocity_error(got[sel], ref, seg)
    assert np.quantile(err, 0.999) < F32_TOL, np.quantile(err, 0.999)
    assert err.max() < 1e-5, err.max()


@pytest.mark.parametrize("data_seed", [1239, 1241])
def test_fused_mixed_precision_tiny_cells(mcc, data_seed):
    """Mixed path on cells of 1 to ~24 particles (species of 0-5: inactive and one-pair interactions, odd triplets,
    inter-species rounds of N_min = 1). The scatter holds 2e-6 for every particle, and the failed corrections equal
    the oracle's. The whole step does not hold 2e-6 here: each species' crossing energy pair
    absorbs the remainder of Delta E_s (Eq. DeltaEs, Eq. U_inelastic), which carries the float kinematics' error of
    the interaction's energy exchange (~1e-7 of it), and in a cell this small that pair is often the species' only
    one, with a CM energy far below the exchanged energy, so the error becomes a large relative change of its two
    velocities (measured: up to 1.9e-4 over three data seeds, the same values as the group kernels gave before their
    instruction-footprint changes). The bound stated for this regime is 5e-4; per-cell conservation before the store
    holds 1e-13 here too (test_fused_conservation_before_store)."""
    wl = W.three_species(n_cells=400, mean_count=4, data_seed=data_seed)
    got, ref, corr, fail, rc, rf = _run_fused(mcc, wl, "f32", n_steps=1, correct=False)
    assert velocity_error(got, ref, wl.offsets).max() < F32_TOL
    got, ref, corr, fail, rc, rf = _run_fused(mcc, wl, "f32", n_steps=1)
    np.testing.assert_array_equal(fail, rf)
    assert velocity_error(got, ref, wl.offsets).max() < 5e-4


@pytest.mark.parametrize("name,make,kw,scatter_max", [
    ("duplicity_weighting", lambda: W.three_species(n_cells=200, mean_count=120), {"weighting": 1}, F32_TOL),
    ("nxn_two_species", lambda: W.equilibration(n_cells=100, mean_count=12, precision="f32"), {"pairing": 1}, 1e-5),
], ids=["duplicity_weighting", "nxn_two_species"])
def test_fused_mixed_precision_options(mcc, name, make, kw, scatter_max):
    """Mixed path with the step's options. Scatter alone: every particle within 2e-6 of the FP64 oracle, except with
    the N x N pairing, where each particle is scattered by every partner in turn and the float rounding of ~N pair
    kinematics accumulates (every particle within 1e-5). Whole step: the bound of test_fused_mixed_precision (99.9%
    within 2e-6, every particle within 1e-5; a crossing energy pair carries the float error of the scatter's energy
    exchange)."""
    wl = make()
    got, ref, corr, fail, rc, rf = _run_fused(mcc, wl, "f32", n_steps=1, correct=False, **dict(kw))
    err = velocity_error(got, ref, wl.offsets)
    assert err.max() < scatter_max, err.max()
    got, ref, corr, fail, rc, rf = _run_fused(mcc, wl, "f32", n_steps=1, **dict(kw))
    err = velocity_error(got, ref, wl.offsets)
    np.testing.assert_array_equal(fail, rf)
    assert np.quantile(err, 0.999) < F32_TOL, np.quantile(err, 0.999)
    assert err.max() < 1e-5, err.max()


def test_graph_of_one_step_serves_every_step(mcc):
    """With the step index in device memory, a CUDA graph captured from one fused step, replayed three times, gives
    exactly the three steps of a direct call, and leaves the counter three steps on."""
    import torch
    wl = W.three_species(n_cells=60, mean_count=90)
    sp = _species(wl)
    v0, w, off = device_state(wl, "f32")
    v1 = [x.clone() for x in v0]
    pp, _ = _params(mcc, wl, step=11)
    mcc.mcc_step_fused(*v0, w, off, wl.n_cells, wl.n_species, sp, wl.lnL, pp, n_steps=3)
    counter = torch.tensor([0], dtype=torch.int64, device="cuda")
    pd, _ = _params(mcc, wl, step=0)
    pd.step_device = counter
    warm = [x.clone() for x in v1]
    mcc.mcc_step_fused(*warm, w, off, wl.n_cells, wl.n_species, sp, wl.lnL, pd, n_steps=1,
                       max_cell=int(wl.counts.sum(1).max()))  # workspaces, warm-up
    torch.cuda.synchronize()
    counter.fill_(11)
    g = torch.cuda.CUDAGraph()
    mc = int(wl.counts.sum(1).max())  # given, so that the captured call does no host read
    with torch.cuda.graph(g):
        mcc.mcc_step_fused(*v1, w, off, wl.n_cells, wl.n_species, sp, wl.lnL, pd, n_steps=1, max_cell=mc)
    for _ in range(3):
        g.replay()
    torch.cuda.synchronize()
    mcc.sync_status(0)
    assert int(counter.item()) == 14
    for a, b in zip(v0, v1):
        np.testing.assert_array_equal(a.cpu().numpy(), b.cpu().numpy())


def test_fused_cells_above_every_class(mcc):
    """Mixed path: cells above the largest group class run on the one-CTA kernel (from its workspace slabs when larger
    than its tile) in the same call. Group capacity 16 per warp (classes up to 256 particles), one-CTA tile 128
    particles, cells of ~300. That kernel keeps float velocities between pairs: its scatter holds 2e-6 for every
    particle; its whole step 2e-6 for 99% of particles (each species' last energy pair absorbs an energy violation
    formed from float-stored velocities)."""
    wl = W.three_species(n_cells=40, mean_count=300)
    ctx = mcc.context(0)
    ctx.set_group_capacity(16, 256)
    ctx.set_tile_cap(128)
    try:
        assert ctx.group_capacities(mcc.F32_MIXED)[-1] == 256
        got, ref, corr, fail, rc, rf = _run_fused(mcc, wl, "f32", n_steps=1, correct=False)
        err_scatter = velocity_error(got, ref, wl.offsets)
        got, ref, corr, fail, rc, rf = _run_fused(mcc, wl, "f32", n_steps=1)
    finally:
        ctx.set_group_capacity(0)
        ctx.set_tile_cap(0)
    assert (wl.counts.sum(1) > 256).sum() > 10
    assert err_scatter.max() < F32_TOL, err_scatter.max()
    err = velocity_error(got, ref, wl.offsets)
    ok = np.repeat(fail == rf, np.diff(wl.offsets[::wl.n_species]))
    assert np.quantile(err[ok], 0.99) < F32_TOL
    assert err[ok].max() < 2e-4


def test_fp64_step_on_one_cta_kernel(mcc):
    """The FP64 path has no group size classes: every cell runs on the one-CTA kernel."""
    assert mcc.context(0).group_capacities(mcc.F64) == [0, 0, 0, 0, 0]


def _philox_top_words(seed, step, cell, inter_tag, n):
    """Top 32 bits of the n permutation keys of a segment: Philox-4x32-10 (Salmon et al., SC'11) evaluated with
    numpy over the counters {i/2, cell, step, tag}; word 0 of the block for even i, word 2 for odd i."""
    mask = np.uint64(0xFFFFFFFF)
    h = np.arange((n + 1) // 2, dtype=np.uint64)
    c = [h, np.full_like(h, cell), np.full_like(h, step & 0xFFFFFFFF), np.full_like(h, inter_tag)]
    k0, k1 = np.uint64(seed & 0xFFFFFFFF), np.uint64(seed >> 32)
    for r in range(10):
        if r:
            k0 = (k0 + np.uint64(0x9E3779B9)) & mask
            k1 = (k1 + np.uint64(0xBB67AE85)) & mask
        p0 = np.uint64(0xD2511F53) * c[0]
        p1 = np.uint64(0xCD9E8D57) * c[2]
        c = [(p1 >> np.uint64(32)) ^ c[1] ^ k0, p1 & mask, (p0 >> np.uint64(32)) ^ c[3] ^ k1, p0 & mask]
    top = np.empty(2 * len(h), dtype=np.uint64)
    top[0::2], top[1::2] = c[0], c[2]
    return top[:n]


def test_permutation_key_tie_in_top_word(mcc):
    """The group kernel's counting sort keys on the top 32 bits of each 64-bit permutation key; two keys equal there
    are ordered by the rest of the key. A cell whose segment holds such a pair (found by search) gives the oracle's
    pairs, so the mixed step matches it (and the FP64 step, on the one-CTA kernel)."""
    seed, step, n = 0x5EED0001, 5, 4000
    found = None
    for cell in range(4000):
        top = _philox_top_words(seed, step, cell, (0 << 8) | 1, n)
        if len(np.unique(top)) < n:
            found = cell
            break
    assert found is not None
    wl = W.isotropisation(n_cells=found + 1, per_cell=2)
    counts = np.full((found + 1, 1), 2, dtype=np.int64)
    counts[found, 0] = n
    rng = np.random.default_rng(11)
    N = int(counts.sum())
    wl.counts = counts
    wl.vx, wl.vy, wl.vz = (rng.normal(0.0, 1.0, N) for _ in range(3))
    wl.w = 10.0 ** rng.uniform(0.0, 1.0, N)
    wl.seed = seed
    for dtype, tol in (("f32", F32_TOL), ("f64", F64_TOL)):
        v, w, off = device_state(wl, dtype)
        st = oracle_state(wl, dtype)
        pp, op = _params(mcc, wl, step=step)
        corr, fail = mcc.mcc_step_fused(*v, w, off, wl.n_cells, wl.n_species, _species(wl), wl.lnL, pp, n_steps=1)
        mcc.sync_status(0)
        rc, rf = O.step(st, wl.q, wl.m, wl.lnL, op, n_steps=1)
        err = velocity_error(gpu_velocities(v), st.v(), wl.offsets)
        assert err.max() < tol, (dtype, err.max())
        np.testing.assert_array_equal(fail.cpu().numpy(), rf)


def test_fused_conservation(mcc):
    """FP64 path: per-cell momentum and energy drift <= 1e-13 relative on the stored state. Mixed path: drift of the
    float-stored state within a few float roundings of the velocities (2^-24 relative per component)."""
    for dtype, tol in (("f64", 1e-13), ("f32", 8 * 2.0 ** -24)):
        wl = W.three_species(n_cells=100, mean_count=200, precision=dtype)
        v, w, off = device_state(wl, dtype)
        v0 = gpu_velocities(v)
        sp = wl.species_of_particles()
        P0, E0, A0 = cell_moments(v0, wl.w, wl.m, sp, wl.offsets, wl.n_cells, wl.n_species)
        pp, _ = _params(mcc, wl)
        corr, fail = mcc.mcc_step_fused(*v, w, off, wl.n_cells, wl.n_species, _species(wl), wl.lnL, pp, n_steps=3)
        mcc.sync_status(0)
        P1, E1, _ = cell_moments(gpu_velocities(v), wl.w, wl.m, sp, wl.offsets, wl.n_cells, wl.n_species)
        assert np.max(np.abs(P1 - P0).max(axis=1) / A0) < tol, dtype
        assert np.max(np.abs(E1 - E0) / E0) < tol, dtype


@pytest.mark.parametrize("name,make", [
    ("three_species", lambda: W.three_species(n_cells=100, mean_count=200)),
    ("three_species_classes", lambda: W.three_species(n_cells=40, mean_count=900)),
    ("relativistic", lambda: W.relativistic_beam(n_cells=60, count_lo=16, count_hi=600)),
    ("three_species_tiny_cells", lambda: W.three_species(n_cells=400, mean_count=4)),
], ids=["three_species", "three_species_classes", "relativistic", "three_species_tiny_cells"])
def test_fused_conservation_before_store(mcc, name, make):
    """Mixed path: per cell, the float-float state the step holds on chip before it stores it conserves momentum and
    kinetic energy to <= 1e-13 relative (Sec. 4; read from the step's residual output): its sums, coefficients and
    energy pairs are FP64-grade although its pair kinematics run in float. (The FP64 path stores what it holds; its
    stored state is checked by test_fused_conservation.)"""
    import torch
    wl = make()
    dtype = "f32"
    v, w, off = device_state(wl, dtype)
    res = torch.full((2 * wl.n_cells,), -1.0, dtype=torch.float64, device="cuda")
    pp, _ = _params(mcc, wl)
    pp.residual = res
    mcc.mcc_step_fused(*v, w, off, wl.n_cells, wl.n_species, _species(wl), wl.lnL, pp, n_steps=1)
    mcc.sync_status(0)
    r = res.cpu().numpy().reshape(-1, 2)
    assert (r >= 0).all()
    assert r[:, 0].max() <= 1e-13, r[:, 0].max()
    assert r[:, 1].max() <= 1e-13, r[:, 1].max()


def test_fail_policy_error_latches(mcc):
    import torch
    v = [torch.tensor(x, dtype=torch.float64, device="cuda") for x in ([1.0, -0.5, 0.0], [0.0, 0.3, -0.4],
                                                                      [0.0, 0.0, 0.7])]
    w = torch.tensor([1e6, 1.0, 1.0], dtype=torch.float64, device="cuda")
    off = torch.tensor([0, 3], dtype=torch.int64, device="cuda")
    seen = False
    for seed in range(200):
        vv = [x.clone() for x in v]
        p = mcc.Params(method=mcc.N97, dt=0.5, seed=seed, fail_policy=mcc.FAIL_ERROR)
        corr, fail = mcc.mcc_step_fused(*vv, w, off, 1, 1, [(-1.0, 1.0)], 10.0, p)
        try:
            mcc.sync_status(0)
        except mcc.MccError as e:
            assert e.code == -5
            assert int(fail[0]) == 1
            seen = True
            break
    assert seen


def test_oversize_cell_latches_bounds(mcc):
    wl = W.equilibration(n_cells=4, mean_count=30, precision="f64")
    v, w, off = device_state(wl, "f64")
    pp, _ = _params(mcc, wl)
    mcc.mcc_step_fused(*v, w, off, wl.n_cells, wl.n_species, _species(wl), wl.lnL, pp, max_cell=8)
    with pytest.raises(mcc.MccError) as e:
        mcc.sync_status(0)
    assert e.value.code == -6


def test_max_cell_above_segment_limit_rejected(mcc):
    """In-cell particle indices are 20-bit key fields: max_cell above MCC_MAX_SEGMENT is refused on the host
    (MCC_ERR_TOO_LARGE) before any work, so a segment past the limit (which mcc_bin_static does not report) can only
    reach the step as a cell above max_cell, which latches MCC_ERR_BOUNDS."""
    wl = W.equilibration(n_cells=4, mean_count=30, precision="f32")
    v, w, off = device_state(wl, "f32")
    pp, _ = _params(mcc, wl)
    with pytest.raises(mcc.MccError) as e:
        mcc.mcc_step_fused(*v, w, off, wl.n_cells, wl.n_species, _species(wl), wl.lnL, pp, max_cell=(1 << 20) + 1)
    assert e.value.code == -7
    mcc.sync_status(0)


def test_invalid_arguments_rejected_on_host(mcc):
    wl = W.equilibration(n_cells=2, mean_count=4, precision="f64")
    v, w, off = device_state(wl, "f64")
    for bad in (dict(dt=-1.0), dict(fE=0.0), dict(fE=1.5), dict(method=7)):
        pp, _ = _params(mcc, wl, **bad)
        with pytest.raises(mcc.MccError) as e:
            mcc.mcc_step_fused(*v, w, off, wl.n_cells, wl.n_species, _species(wl), wl.lnL, pp)
        assert e.value.code == -1


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_resume_from_saved_state_is_bit_exact(mcc, dtype):
    """Checkpoint / resume: the state is (velocities, weights, step, seed) because every draw is keyed by the step, so
    two steps, a copy of the state to the host and back, and two more steps give exactly four uninterrupted steps."""
    import torch
    wl = W.three_species(n_cells=50, mean_count=90, precision=dtype)
    sp = _species(wl)
    v, w, off = device_state(wl, dtype)
    ref = [x.clone() for x in v]
    pp, _ = _params(mcc, wl, step=20)
    mcc.mcc_step_fused(*ref, w, off, wl.n_cells, wl.n_species, sp, wl.lnL, pp, n_steps=4)
    mcc.mcc_step_fused(*v, w, off, wl.n_cells, wl.n_species, sp, wl.lnL, pp, n_steps=2)
    saved = [x.cpu().numpy().copy() for x in v]
    restored = [torch.from_numpy(x).cuda() for x in saved]
    pr, _ = _params(mcc, wl, step=22)
    mcc.mcc_step_fused(*restored, w, off, wl.n_cells, wl.n_species, sp, wl.lnL, pr, n_steps=2)
    mcc.sync_status(0)
    for a, b in zip(ref, restored):
        np.testing.assert_array_equal(a.cpu().numpy(), b.cpu().numpy())
