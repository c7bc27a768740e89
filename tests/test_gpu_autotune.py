"""The autotuner on the GPU: it times its candidates on a scratch copy (the caller's state is unchanged), applies the
winner to the context, and a second call is served from the persistent cache."""
import numpy as np
import pytest

from paper_2407_19151_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def test_autotune_applies_and_caches(tmp_path, monkeypatch):
    import torch

    import paper_2407_19151_gb300 as mcc
    mcc.build()
    monkeypatch.setenv("MCC_AUTOTUNE_CACHE", str(tmp_path / "autotune.json"))
    wl = W.three_species(n_cells=400, mean_count=400).weight_ordered()
    v = [torch.from_numpy(np.ascontiguousarray(x)).cuda() for x in (wl.vx, wl.vy, wl.vz)]
    w = torch.from_numpy(wl.w).cuda()
    off = torch.from_numpy(wl.offsets).cuda()
    sp = list(zip(wl.q.tolist(), wl.m.tolist()))
    p = mcc.Params(method=wl.method, dt=wl.dt, fE=wl.fE, seed=wl.seed)
    mc = int(wl.counts.sum(1).max())
    before = [x.clone() for x in v]
    ctx = mcc.context(0)
    try:
        r1 = mcc.autotune(*v, w, off, wl.n_cells, wl.n_species, sp, wl.lnL, p, mc)
        assert not r1["cached"] and r1["ms"] is not None and r1["ms"] > 0
        for a, b in zip(v, before):
            assert torch.equal(a, b)  # timed on a scratch copy
        caps_tuned = ctx.group_capacities(mcc.F32_MIXED)
        ctx.set_group_capacity(0)
        ctx.set_group_capacity(r1["group_cap"])
        assert ctx.group_capacities(mcc.F32_MIXED) == caps_tuned
        import importlib
        T = importlib.import_module("paper_2407_19151_gb300.autotune")
        T._CACHE.clear()  # the second call must come from the file
        r2 = mcc.autotune(*v, w, off, wl.n_cells, wl.n_species, sp, wl.lnL, p, mc)
        assert r2["cached"] and r2["group_cap"] == r1["group_cap"] and r2["tile_cap"] == r1["tile_cap"]
        assert (tmp_path / "autotune.json").exists()
    finally:
        ctx.set_group_capacity(0)
        ctx.set_tile_cap(0)
    mcc.sync_status(0)
