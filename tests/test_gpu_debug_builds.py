"""The debugging builds of the library, each loaded in a child process (one library per process): the bounds-checked
build (every index of the group kernels checked against its bound) runs the mixed fused step with no violation
recorded and the oracle's results, and the phase-timing build reports cycles for every phase of every launched size
class. A third case plants an oversize cell (more particles than max_cell) to show that the bound check latches
MCC_ERR_BOUNDS on the host-visible status without a fault."""
import json
import os
import subprocess
import sys
import textwrap

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

_CHILD = textwrap.dedent('''
    import json, sys
    import numpy as np, torch
    sys.path.insert(0, ROOT)
    sys.path.insert(0, ROOT + "/tests")
    import paper_2407_19151_gb300 as mcc
    from paper_2407_19151_gb300 import workloads as W
    import oracle as O
    from _parity import velocity_error
    lib = mcc.lib()
    out = {"bounds_build": lib.mcc_debug_bounds_build(), "clocks_build": lib.mcc_phase_clocks_build()}
    wl = W.three_species(n_cells=200, mean_count=500).weight_ordered()
    dev = "cuda:0"
    v = [torch.from_numpy(np.asarray(x, dtype=np.float32)).to(dev) for x in (wl.vx, wl.vy, wl.vz)]
    w = torch.from_numpy(wl.w).to(dev)
    off = torch.from_numpy(wl.offsets).to(dev)
    sp = list(zip(wl.q.tolist(), wl.m.tolist()))
    mc = int(wl.counts.sum(1).max())
    kw = dict(method=wl.method, dt=wl.dt, fE=wl.fE, seed=wl.seed, step=3)
    ctx = mcc.context(0)
    mcc.mcc_step_fused(*v, w, off, wl.n_cells, wl.n_species, sp, wl.lnL, mcc.Params(**kw), n_steps=1, max_cell=mc)
    out["status"] = ctx.sync_status()
    out["record"] = ctx.debug_record()
    out["clocks"] = ctx.phase_clocks()
    got = np.stack([x.double().cpu().numpy() for x in v], 1)
    st = O.State(*[np.asarray(x, dtype=np.float32).astype(np.float64) for x in (wl.vx, wl.vy, wl.vz)], wl.w,
                 wl.offsets, wl.n_cells, wl.n_species)
    O.step(st, wl.q, wl.m, wl.lnL, O.Params(**kw))
    out["err_p999"] = float(np.quantile(velocity_error(got, st.v(), wl.offsets), 0.999))
    # a cell above max_cell: the group kernels' bound check latches MCC_ERR_BOUNDS and skips it
    mcc.mcc_step_fused(*v, w, off, wl.n_cells, wl.n_species, sp, wl.lnL, mcc.Params(**kw), n_steps=1, max_cell=mc - 1)
    out["oversize_status"] = ctx.sync_status()
    print(json.dumps(out))
''')


def _run_child(lib_path):
    env = dict(os.environ, MCC_LIBRARY=lib_path)
    r = subprocess.run([sys.executable, "-c", f"ROOT = {ROOT!r}\n" + _CHILD], env=env, capture_output=True,
                       text=True, timeout=900, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-3000:]
    return json.loads(r.stdout.strip().splitlines()[-1])


def test_bounds_checked_build():
    from paper_2407_19151_gb300 import _build
    out = _run_child(_build.build(debug_bounds=True))
    assert out["bounds_build"] == 1 and out["clocks_build"] == 0
    assert out["status"] == 0
    assert out["record"] == [0, 0, 0, 0], out["record"]
    assert out["err_p999"] < 2e-6, out["err_p999"]
    assert out["oversize_status"] == -6  # MCC_ERR_BOUNDS, latched on the device, read on the host


def test_phase_clock_build():
    from paper_2407_19151_gb300 import _build
    out = _run_child(_build.build(phase_clocks=True))
    assert out["clocks_build"] == 1 and out["bounds_build"] == 0
    assert out["status"] == 0
    launched = [k for k in range(5) if out["clocks"][k][7] > 0]
    assert launched, out["clocks"]
    assert sum(out["clocks"][k][7] for k in range(5)) == 200  # every cell visited once
    for k in launched:
        assert all(c > 0 for c in out["clocks"][k][:7]), (k, out["clocks"][k])
    assert out["err_p999"] < 2e-6
