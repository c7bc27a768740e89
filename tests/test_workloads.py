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


def test_grid_dims_factorise_the_cells():
    for n in (1, 7, 60, 200, 4096, 1 << 18):
        nx, ny, nz = W.grid_dims(n)
        assert nx * ny * nz == n and nx >= ny >= 1 and nz >= 1
    assert W.grid_dims(1 << 18) == (64, 64, 64)


def test_pic_setup_places_each_particle_in_its_own_cell():
    for wl in (W.three_species(n_cells=60, mean_count=40), W.relativistic_beam(n_cells=24, count_lo=16,
                                                                               count_hi=64)):
        grid, x, y, z, dt_push = W.pic_setup(wl, cfl=0.3)
        (nx, ny, nz), (lx, ly, lz) = grid
        assert (lx, ly, lz) == (nx, ny, nz)   # unit cells
        dtype = np.float32 if wl.precision == "f32" else np.float64
        assert x.dtype == dtype and len(x) == wl.n
        cell = np.floor(x).astype(int) + nx * (np.floor(y).astype(int) + ny * np.floor(z).astype(int))
        np.testing.assert_array_equal(cell, wl.cell_of_particles())
        if wl.relativistic:
            assert dt_push == 0.3 / wl.c
        else:
            e = wl.species_of_particles() == int(np.argmin(wl.m))
            assert abs(dt_push * np.sqrt(np.mean(np.asarray(wl.vx, np.float64)[e] ** 2)) - 0.3) < 1e-12


def test_pic_loop_rejects_unknown_order():
    import pytest
    from paper_2407_19151_gb300.pic import PicLoop
    with pytest.raises(ValueError):
        PicLoop(*([None] * 9), 1, 1, None, [], 1.0, None, 0.1, order="sorted")
