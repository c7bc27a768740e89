"""The allocation-free cell sort, mcc_bin_static, for callers that cannot allocate device memory: called through
the C ABI (ctypes, plain device pointers) twice in a row on different inputs, each result bit-identical to
mcc_bin's. Integers, so the tolerance is exact equality. Collected last so that a stop at the first failure has
already run every other test; it passes alone in a fresh process as well as after the others."""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _inputs(seed, n, n_cells, n_species):
    rng = np.random.default_rng(seed)
    return rng.integers(0, n_cells, n).astype(np.int32), rng.integers(0, n_species, n).astype(np.int32)


def test_bin_static_matches_bin_twice():
    import torch

    import paper_2407_19151_gb300 as mcc

    mcc.build()
    lib = mcc.lib()
    stream = C.c_void_p(torch.cuda.current_stream(0).cuda_stream)
    # small segments; segments above the one-CTA sort's shared-memory capacity (8 cells, about 25k particles each);
    # exactly MCC_BIN_STATIC_MAX_KEYS segments; no particles
    for seed, n, n_cells, n_species in [(1, 300_000, 4096, 3), (2, 50_000, 777, 2), (3, 200_000, 8, 1),
                                        (4, 3_000_000, 1 << 20, 2), (5, 0, 10, 2)]:
        cell, sp = _inputs(seed, n, n_cells, n_species)
        d_cell, d_sp = torch.from_numpy(cell).cuda(), torch.from_numpy(sp).cuda()
        perm = torch.empty(n, dtype=torch.int32, device="cuda")
        offsets = torch.empty(n_cells * n_species + 1, dtype=torch.int64, device="cuda")
        rc = lib.mcc_bin_static(C.c_void_p(d_cell.data_ptr()), C.c_void_p(d_sp.data_ptr()), n, n_cells, n_species,
                                C.c_void_p(perm.data_ptr()), C.c_void_p(offsets.data_ptr()), stream)
        assert rc == 0
        torch.cuda.synchronize()
        ref_perm, ref_off = mcc.mcc_bin(d_cell, d_sp, n_cells, n_species)
        mcc.sync_status(0)
        np.testing.assert_array_equal(offsets.cpu().numpy(), ref_off.cpu().numpy())
        np.testing.assert_array_equal(perm.cpu().numpy(), ref_perm.cpu().numpy())


def test_bin_static_rejects_too_many_segments():
    import torch

    import paper_2407_19151_gb300 as mcc

    lib = mcc.lib()
    d = torch.zeros(4, dtype=torch.int32, device="cuda")
    offsets = torch.empty(8, dtype=torch.int64, device="cuda")
    rc = lib.mcc_bin_static(C.c_void_p(d.data_ptr()), C.c_void_p(d.data_ptr()), 4, (1 << 21) + 1, 1,
                            C.c_void_p(d.data_ptr()), C.c_void_p(offsets.data_ptr()), None)
    assert rc == -7


def test_bin_static_wrapper_preallocated():
    """The Python wrapper with caller-owned outputs, on the tensors' device made current by the wrapper."""
    import torch

    import paper_2407_19151_gb300 as mcc

    cell, sp = _inputs(6, 120_000, 300, 3)
    d_cell, d_sp = torch.from_numpy(cell).cuda(), torch.from_numpy(sp).cuda()
    perm = torch.empty(cell.size, dtype=torch.int32, device="cuda")
    offsets = torch.empty(300 * 3 + 1, dtype=torch.int64, device="cuda")
    p, o = mcc.mcc_bin_static(d_cell, d_sp, 300, 3, perm=perm, offsets=offsets)
    assert p.data_ptr() == perm.data_ptr() and o.data_ptr() == offsets.data_ptr()
    ref_perm, ref_off = mcc.mcc_bin(d_cell, d_sp, 300, 3)
    mcc.sync_status(0)
    np.testing.assert_array_equal(offsets.cpu().numpy(), ref_off.cpu().numpy())
    np.testing.assert_array_equal(perm.cpu().numpy(), ref_perm.cpu().numpy())
