"""The host-buffer pipeline (cell chunks copied in, stepped and copied out on three streams) gives exactly the
result of the same steps on a device-resident state: random draws are keyed by the global cell id."""
import numpy as np
import pytest

from paper_2407_19151_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("chunks,buffers", [(1, 1), (4, 2), (7, 3)])
def test_step_host_equals_device_steps(chunks, buffers):
    import torch

    import paper_2407_19151_gb300 as mcc
    from paper_2407_19151_gb300.host_pipeline import step_host
    mcc.build()
    wl = W.three_species(n_cells=300, mean_count=120)
    sp = list(zip(wl.q.tolist(), wl.m.tolist()))
    p = mcc.Params(method=wl.method, dt=wl.dt, fE=wl.fE, seed=wl.seed, step=5)
    v = [torch.from_numpy(np.ascontiguousarray(x)).cuda() for x in (wl.vx, wl.vy, wl.vz)]
    w = torch.from_numpy(wl.w).cuda()
    off = torch.from_numpy(wl.offsets).cuda()
    corr, fail = mcc.mcc_step_fused(*v, w, off, wl.n_cells, wl.n_species, sp, wl.lnL, p, n_steps=2)
    mcc.sync_status(0)
    host = [torch.from_numpy(np.ascontiguousarray(x)).pin_memory() for x in (wl.vx, wl.vy, wl.vz)]
    hw = torch.from_numpy(wl.w).pin_memory()
    hc, hf = step_host(*host, hw, wl.offsets, wl.n_cells, wl.n_species, sp, wl.lnL, p, n_steps=2, chunks=chunks,
                       buffers=buffers)
    mcc.sync_status(0)
    for a, b in zip(host, v):
        np.testing.assert_array_equal(a.numpy(), b.cpu().numpy())
    np.testing.assert_array_equal(hc, corr.cpu().numpy())
    np.testing.assert_array_equal(hf, fail.cpu().numpy())


@pytest.mark.parametrize("chunks,buffers", [(4, 2), (5, 3)])
def test_step_host_round_trips(chunks, buffers):
    """Three round trips through host memory of one step each (the pipeline kept full across round trips) equal three
    device-resident steps, and the counters accumulate over them."""
    import torch

    import paper_2407_19151_gb300 as mcc
    from paper_2407_19151_gb300.host_pipeline import step_host
    mcc.build()
    wl = W.three_species(n_cells=240, mean_count=150).weight_ordered()
    sp = list(zip(wl.q.tolist(), wl.m.tolist()))
    p = mcc.Params(method=wl.method, dt=wl.dt * 5, fE=wl.fE, seed=wl.seed, step=11)
    v = [torch.from_numpy(np.ascontiguousarray(x)).cuda() for x in (wl.vx, wl.vy, wl.vz)]
    w = torch.from_numpy(wl.w).cuda()
    off = torch.from_numpy(wl.offsets).cuda()
    corr, fail = mcc.mcc_step_fused(*v, w, off, wl.n_cells, wl.n_species, sp, wl.lnL, p, n_steps=3)
    mcc.sync_status(0)
    host = [torch.from_numpy(np.ascontiguousarray(x)).pin_memory() for x in (wl.vx, wl.vy, wl.vz)]
    hw = torch.from_numpy(wl.w).pin_memory()
    hc, hf = step_host(*host, hw, wl.offsets, wl.n_cells, wl.n_species, sp, wl.lnL, p, n_steps=1, chunks=chunks,
                       buffers=buffers, round_trips=3)
    mcc.sync_status(0)
    for a, b in zip(host, v):
        np.testing.assert_array_equal(a.numpy(), b.cpu().numpy())
    np.testing.assert_array_equal(hc, corr.cpu().numpy())
    np.testing.assert_array_equal(hf, fail.cpu().numpy())
