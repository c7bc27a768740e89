"""Host-side input layout: the weight-ordered copy of a workload keeps every particle and its cell and species."""
import numpy as np

from paper_2407_19151_gb300 import workloads as W


def test_weight_ordered_layout():
    wl = W.three_species(n_cells=50, mean_count=60)
    wo = wl.weight_ordered()
    off = wl.offsets
    np.testing.assert_array_equal(wo.offsets, off)
    for k in range(len(off) - 1):
        a, b = off[k], off[k + 1]
        assert np.all(np.diff(wo.w[a:b]) <= 0)
        # the same particles (weight and velocity together), only reordered within the segment
        before = sorted(zip(wl.w[a:b], wl.vx[a:b], wl.vy[a:b], wl.vz[a:b]))
        after = sorted(zip(wo.w[a:b], wo.vx[a:b], wo.vy[a:b], wo.vz[a:b]))
        assert before == after


def test_weight_ordered_keeps_equal_weights_in_place():
    wl = W.equilibration(n_cells=3, mean_count=20)   # electrons all have weight 1
    wo = wl.weight_ordered()
    off = wl.offsets
    a, b = off[0], off[1]
    np.testing.assert_array_equal(wo.vx[a:b], wl.vx[a:b])
