"""Multi-GPU sharding: contiguous, particle-balanced cell ranges; world-size-2 gloo runs on CPU in which each rank
steps its shard and the gathered result equals the unsharded run bit for bit while the per-species diagnostics are
combined with an all-reduce (once with the ranks written out by hand, once through the product's ShardedStep with
the oracle as its device side); on the GPU, ShardedStep against the whole-problem step and the species-moments
kernel against the same sums on the host."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle as O
from paper_2407_19151_gb300 import Params, sharding
from paper_2407_19151_gb300 import workloads as W


def test_shard_cells_cover_and_balance():
    wl = W.three_species(n_cells=1000, mean_count=64)
    off = wl.offsets
    for world in (1, 2, 3, 7):
        ranges = [sharding.shard_cells(off, 3, world, r) for r in range(world)]
        assert ranges[0][0] == 0 and ranges[-1][1] == wl.n_cells
        for (a, b), (c, d) in zip(ranges, ranges[1:]):
            assert b == c and a <= b
        sizes = [off[b * 3] - off[a * 3] for a, b in ranges]
        assert max(sizes) - min(sizes) <= 2 * int(wl.counts.sum(1).max())


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank_main(rank, world, port, out_dir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    wl = W.equilibration(n_cells=40, mean_count=30, precision="f64")
    c0, c1 = sharding.shard_cells(wl.offsets, 2, world, rank)
    st = O.State(wl.vx, wl.vy, wl.vz, wl.w, wl.offsets, wl.n_cells, 2)
    p = O.Params(method=wl.method, dt=wl.dt * 5, seed=wl.seed, step=4)
    O.step(st, wl.q, wl.m, wl.lnL, p, n_steps=2, cell_begin=c0, cell_end=c1)
    _, p0, p1 = sharding.shard_view(wl.offsets, 2, c0, c1)
    mine = torch.from_numpy(np.stack([st.vx[p0:p1], st.vy[p0:p1], st.vz[p0:p1]], axis=1).copy())
    sizes = [torch.zeros(1, dtype=torch.int64) for _ in range(world)]
    dist.all_gather(sizes, torch.tensor([mine.shape[0]]))
    parts = [torch.zeros((int(n), 3), dtype=torch.float64) for n in sizes]
    _gather_uneven(parts, mine, rank, world)
    diag = torch.from_numpy(sharding.species_moments(st.vx[p0:p1], st.vy[p0:p1], st.vz[p0:p1], wl.w[p0:p1],
                                                     sharding.shard_view(wl.offsets, 2, c0, c1)[0], c1 - c0, 2,
                                                     wl.m))
    dist.all_reduce(diag)
    if rank == 0:
        np.save(os.path.join(out_dir, "gathered.npy"), torch.cat(parts).numpy())
        np.save(os.path.join(out_dir, "diag.npy"), diag.numpy())
    dist.barrier()
    dist.destroy_process_group()


def _gather_uneven(parts, mine, rank, world):
    for r in range(world):
        buf = mine if r == rank else parts[r]
        dist.broadcast(buf, src=r)
        parts[r].copy_(buf)


def test_two_rank_gloo_sharded_step_equals_unsharded(tmp_path):
    O.build()
    world = 2
    mp.spawn(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    got = np.load(tmp_path / "gathered.npy")
    diag = np.load(tmp_path / "diag.npy")
    wl = W.equilibration(n_cells=40, mean_count=30, precision="f64")
    st = O.State(wl.vx, wl.vy, wl.vz, wl.w, wl.offsets, wl.n_cells, 2)
    O.step(st, wl.q, wl.m, wl.lnL, O.Params(method=wl.method, dt=wl.dt * 5, seed=wl.seed, step=4), n_steps=2)
    np.testing.assert_array_equal(got, st.v())
    ref = sharding.species_moments(st.vx, st.vy, st.vz, wl.w, wl.offsets, wl.n_cells, 2, wl.m)
    np.testing.assert_allclose(diag, ref, rtol=1e-13, atol=1e-13 * np.abs(ref).max())


class _OracleShard:
    """The five device-side calls of ShardedStep on the CPU oracle: the global state is kept, the rank's cells are
    stepped with the oracle's cell range (draws keyed by the global cell id), moments over the rank's particles."""

    def __init__(self, q, m):
        self.q, self.m = q, m

    def load(self, vx, vy, vz, w, view):
        return {"st": O.State(vx, vy, vz, w, _GLOBAL["offsets"], _GLOBAL["n_cells"], _GLOBAL["S"]), "view": view}

    def zeros(self, n):
        return np.zeros(max(n, 1), dtype=np.int64)

    def step(self, st, n_cells, S, species, lnL, params, n_steps, max_cell, fail):
        _, _, _, c0, c1 = st["view"]
        p = O.Params(method=params.method, dt=params.dt, fE=params.fE, seed=params.seed, step=params.step)
        _, f = O.step(st["st"], self.q, self.m, lnL, p, n_steps=n_steps, cell_begin=c0, cell_end=c1)
        fail[:c1 - c0] += f[c0:c1]

    def moments(self, st, n_cells, S, species, params, fail):
        local, p0, p1, _, _ = st["view"]
        g = st["st"]
        mom = sharding.species_moments(g.vx[p0:p1], g.vy[p0:p1], g.vz[p0:p1], g.w[p0:p1], local, n_cells, S, self.m)
        cnt = np.diff(local).reshape(n_cells, S).sum(0)
        out = np.concatenate([np.concatenate([mom, cnt[:, None]], axis=1).ravel(), [fail[:n_cells].sum()]])
        return torch.from_numpy(out.astype(np.float64))

    def velocities(self, st):
        _, p0, p1, _, _ = st["view"]
        return st["st"].v()[p0:p1]


_GLOBAL = {}


def _product_rank_main(rank, world, port, out_dir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    wl = W.equilibration(n_cells=40, mean_count=30, precision="f64")
    _GLOBAL.update(offsets=wl.offsets, n_cells=wl.n_cells, S=2)
    params = Params(method=wl.method, dt=wl.dt * 5, seed=wl.seed, step=4)
    sh = sharding.ShardedStep(wl.offsets, wl.n_cells, 2, list(zip(wl.q, wl.m)), wl.lnL, params,
                              backend=_OracleShard(wl.q, wl.m)).load(wl.vx, wl.vy, wl.vz, wl.w)
    assert (sh.c0, sh.c1) == sharding.shard_cells(wl.offsets, 2, world, rank)
    sh.step(1)
    diag, fails = sh.step(1)
    assert sh.params.step == 6 and sh.params.cell_base == sh.c0
    mine = torch.from_numpy(np.ascontiguousarray(sh.velocities()))
    sizes = [torch.zeros(1, dtype=torch.int64) for _ in range(world)]
    dist.all_gather(sizes, torch.tensor([mine.shape[0]]))
    parts = [torch.zeros((int(n), 3), dtype=torch.float64) for n in sizes]
    _gather_uneven(parts, mine, rank, world)
    if rank == 0:
        np.save(os.path.join(out_dir, "gathered.npy"), torch.cat(parts).numpy())
        np.save(os.path.join(out_dir, "diag.npy"), diag)
        np.save(os.path.join(out_dir, "fails.npy"), np.array([fails]))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_gloo_product_sharded_step(tmp_path):
    """ShardedStep on two gloo ranks (the oracle as its device side): each rank owns its cell range, two calls of
    step() advance the step index, the gathered velocities equal two unsharded steps bit for bit, and the
    all-reduced diagnostics equal the whole state's sums."""
    O.build()
    world = 2
    mp.spawn(_product_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    got = np.load(tmp_path / "gathered.npy")
    diag = np.load(tmp_path / "diag.npy")
    wl = W.equilibration(n_cells=40, mean_count=30, precision="f64")
    st = O.State(wl.vx, wl.vy, wl.vz, wl.w, wl.offsets, wl.n_cells, 2)
    p = O.Params(method=wl.method, dt=wl.dt * 5, seed=wl.seed, step=4)
    _, f1 = O.step(st, wl.q, wl.m, wl.lnL, p, n_steps=1)
    _, f2 = O.step(st, wl.q, wl.m, wl.lnL, O.Params(**{**p.__dict__, "step": 5}), n_steps=1)
    np.testing.assert_array_equal(got, st.v())
    ref = sharding.species_moments(st.vx, st.vy, st.vz, wl.w, wl.offsets, wl.n_cells, 2, wl.m)
    np.testing.assert_allclose(diag[:, :5], ref, rtol=1e-13, atol=1e-13 * np.abs(ref).max())
    np.testing.assert_array_equal(diag[:, 5], wl.counts.sum(0))
    assert int(np.load(tmp_path / "fails.npy")[0]) == int(f1.sum() + f2.sum())


@pytest.mark.gpu
@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("rel", [False, True])
def test_species_moments_kernel(dtype, rel):
    """mcc_species_moments against the same sums on the host (FP64), with and without failure counts."""
    import paper_2407_19151_gb300 as mcc
    mcc.build()
    wl = W.relativistic_beam(n_cells=300, count_lo=4, count_hi=400, precision=dtype) if rel else \
        W.three_species(n_cells=500, mean_count=60, precision=dtype)
    tdt = torch.float64 if dtype == "f64" else torch.float32
    v = [torch.from_numpy(np.asarray(x)).to("cuda", tdt) for x in (wl.vx, wl.vy, wl.vz)]
    w = torch.from_numpy(wl.w).cuda()
    off = torch.from_numpy(wl.offsets).cuda()
    fail = torch.arange(wl.n_cells, dtype=torch.int32, device="cuda") % 3
    out = mcc.mcc_species_moments(*v, w, off, wl.n_cells, wl.n_species, list(zip(wl.q, wl.m)), rel, wl.c,
                                  fail).cpu().numpy()
    mcc.sync_status(0)
    vh = [x.double().cpu().numpy() for x in v]
    S = wl.n_species
    sp = np.repeat(np.tile(np.arange(S), wl.n_cells), np.diff(wl.offsets))
    mw = wl.m[sp] * wl.w
    v2 = vh[0] ** 2 + vh[1] ** 2 + vh[2] ** 2
    ke = mw * v2 / (np.sqrt(1 + v2 / wl.c ** 2) + 1) if rel else 0.5 * mw * v2
    for s in range(S):
        sel = sp == s
        want = [wl.w[sel].sum()] + [(mw[sel] * vh[d][sel]).sum() for d in range(3)] + [ke[sel].sum(), sel.sum()]
        scale = [abs(want[0]), (mw[sel] * np.sqrt(v2[sel])).sum(), (mw[sel] * np.sqrt(v2[sel])).sum(),
                 (mw[sel] * np.sqrt(v2[sel])).sum(), abs(want[4]), 1.0]
        for k in range(6):
            assert abs(out[6 * s + k] - want[k]) <= 1e-12 * scale[k], (s, k, out[6 * s + k], want[k])
    assert out[6 * S] == fail.sum().item()


@pytest.mark.gpu
def test_sharded_step_single_rank_equals_whole_run():
    """Without a process group ShardedStep is the whole problem on one GPU: its velocities equal mcc_step_fused on
    the whole state bit for bit, its diagnostics the host sums of the result."""
    import paper_2407_19151_gb300 as mcc
    mcc.build()
    wl = W.three_species(n_cells=80, mean_count=90, precision="f32")
    sp = list(zip(wl.q, wl.m))
    params = mcc.Params(method=wl.method, dt=wl.dt, seed=wl.seed, step=2)
    sh = sharding.ShardedStep(wl.offsets, wl.n_cells, 3, sp, wl.lnL, params).load(wl.vx, wl.vy, wl.vz, wl.w)
    diag, fails = sh.step(2)
    whole = [torch.from_numpy(np.asarray(x)).cuda() for x in (wl.vx, wl.vy, wl.vz)]
    mcc.mcc_step_fused(*whole, torch.from_numpy(wl.w).cuda(), torch.from_numpy(wl.offsets).cuda(), wl.n_cells, 3,
                       sp, wl.lnL, mcc.Params(method=wl.method, dt=wl.dt, seed=wl.seed, step=2), n_steps=2)
    mcc.sync_status(0)
    got = sh.velocities()
    np.testing.assert_array_equal(got, torch.stack(whole, 1).double().cpu().numpy())
    ref = sharding.species_moments(got[:, 0], got[:, 1], got[:, 2], wl.w, wl.offsets, wl.n_cells, 3, wl.m)
    np.testing.assert_allclose(diag[:, :5], ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max())
    assert fails == 0


@pytest.mark.gpu
def test_serial_gpu_shards_equal_whole_run():
    """The CUDA step on two cell shards (rebased offsets, cell_base = first global cell) equals the whole run."""
    import paper_2407_19151_gb300 as mcc
    mcc.build()
    wl = W.three_species(n_cells=60, mean_count=90, precision="f64")
    dev = "cuda:0"
    sp = list(zip(wl.q, wl.m))
    whole = [torch.from_numpy(x.copy()).to(dev) for x in (wl.vx, wl.vy, wl.vz)]
    w = torch.from_numpy(wl.w).to(dev)
    mcc.mcc_step_fused(*whole, w, torch.from_numpy(wl.offsets).to(dev), wl.n_cells, 3, sp, wl.lnL,
                       mcc.Params(method=wl.method, dt=wl.dt, seed=wl.seed, step=2), n_steps=2)
    parts = []
    for r in range(2):
        c0, c1 = sharding.shard_cells(wl.offsets, 3, 2, r)
        loff, p0, p1 = sharding.shard_view(wl.offsets, 3, c0, c1)
        v = [torch.from_numpy(x[p0:p1].copy()).to(dev) for x in (wl.vx, wl.vy, wl.vz)]
        mcc.mcc_step_fused(*v, w[p0:p1].contiguous(), torch.from_numpy(loff).to(dev), c1 - c0, 3, sp, wl.lnL,
                           mcc.Params(method=wl.method, dt=wl.dt, seed=wl.seed, step=2, cell_base=c0), n_steps=2)
        parts.append(torch.stack(v, 1))
    mcc.sync_status(0)
    np.testing.assert_array_equal(torch.cat(parts).cpu().numpy(), torch.stack(whole, 1).cpu().numpy())
