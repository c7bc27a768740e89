"""Host logic of bench.py (no GPU): the size-class table behind the dominant kernel's roofline, the issue ceiling,
and the workload description both arms print."""
import numpy as np

import bench
from paper_2407_19151_gb300 import workloads as W


def test_class_table_partitions_cells_and_particles():
    wl = W.three_species(n_cells=3000, mean_count=600)
    caps = [286, 572, 1144, 2288, 5237]
    ms = np.array([1.0, 2.0, 3.0, 4.0, 5.0, 0.0])
    rows = bench.class_table(wl, caps, ms, 6767.1)
    n = wl.counts.sum(1)
    assert sum(r["cells"] for r in rows) == wl.n_cells
    assert sum(r["particles"] for r in rows) == wl.n
    lo = [0] + caps
    for k, r in enumerate(rows[:5]):  # class k: cells with caps[k-1] < n <= caps[k]
        sel = (n > lo[k]) & (n <= caps[k])
        assert r["cells"] == int(sel.sum()) and r["particles"] == int(n[sel].sum())
        if r["particles"]:
            assert abs(r["achieved_gbs"] - 32 * r["particles"] / (ms[k] * 1e-3) / 1e9) < 1e-9 * r["achieved_gbs"]
    assert rows[5]["cells"] == int((n > caps[-1]).sum())


def test_issue_ceiling():
    dom = {"kernel": "k", "particles": 1_000_000, "ms": 2.0}
    entry = {"kernel": "k", "warp_instructions_per_particle_step": 100.0}
    r = bench.issue_ceiling(entry, dom, 2000.0, 6767.1)
    rate = 152 * 4 * 2000e6
    assert abs(r["floor_ms"] - 100.0 * 1e6 / rate * 1e3) < 1e-12
    assert abs(r["frac"] - r["floor_ms"] / 2.0) < 1e-12
    assert bench.issue_ceiling(dict(entry, kernel="other"), dom, 2000.0, 6767.1) is None
    assert bench.issue_ceiling(None, dom, 2000.0, 6767.1) is None


def test_both_arms_describe_the_same_workload():
    wl = W.three_species(n_cells=500).weight_ordered()
    a = bench.bench_config(wl, "weight_ordered", 1)
    b = bench.bench_config(wl, "weight_ordered", 1)
    assert a == b and a["workload"] == "three_species" and a["n_particles"] == wl.n
    assert a["pairs_per_step"] == wl.pairs_per_step()
