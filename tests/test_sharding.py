"""Multi-GPU sharding logic on CPU: contiguous, particle-balanced cell ranges, and a world-size-2 gloo run in which
each rank steps its shard (oracle, global cell ids) and the gathered result equals the unsharded run bit for bit;
the per-species diagnostics are combined with an all-reduce."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle as O
from paper_2407_19151_gb300 import sharding
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
