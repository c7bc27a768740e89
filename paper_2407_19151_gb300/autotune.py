"""Project autotuner for the fused step: picks the on-chip tile (particles staged in shared memory per cell; larger
cells run from workspace slabs), which sets how many cells each SM holds at once.

Each candidate is timed on one fused step over a scratch copy of the velocities (the caller's state is untouched),
with CUDA events on the current stream, after one untimed step. The winner is cached per (device, precision,
relativistic, cells, largest cell) and applied to the context with mcc_set_tile_cap.
"""
from __future__ import annotations

import torch

from . import _binding as B

_CACHE: dict[tuple, int] = {}
CANDIDATES = (0, 128, 192, 256, 384, 512, 768, 1024, 1536, 2048, 3072, 4096)


def autotune_tile_cap(vx, vy, vz, w, offsets, n_cells: int, n_species: int, species, lnL, params: B.Params,
                      max_cell: int, interactions=None, candidates=CANDIDATES, verbose: bool = False) -> int:
    ctx = B.context(vx.device)
    key = (vx.device.index, vx.dtype, bool(params.relativistic), int(n_cells), int(max_cell))
    if key in _CACHE:
        ctx.set_tile_cap(_CACHE[key])
        return _CACHE[key]
    scratch = [x.clone() for x in (vx, vy, vz)]
    corr = torch.zeros(max(n_cells, 1), dtype=torch.int32, device=vx.device)
    fail = torch.zeros_like(corr)
    stream = torch.cuda.current_stream(vx.device)
    seen = set()
    best, best_ms = 0, float("inf")
    for cap in candidates:
        eff = min(cap, max_cell) if cap else 0
        if eff in seen:
            continue
        seen.add(eff)
        ctx.set_tile_cap(eff)
        try:
            B.mcc_step_fused(*scratch, w, offsets, n_cells, n_species, species, lnL, params, 1, max_cell,
                             interactions, corr, fail)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            B.mcc_step_fused(*scratch, w, offsets, n_cells, n_species, species, lnL, params, 1, max_cell,
                             interactions, corr, fail)
            e1.record(stream)
            torch.cuda.synchronize(vx.device)
        except B.MccError:
            continue
        ms = e0.elapsed_time(e1)
        if verbose:
            print(f"autotune tile {eff or 'auto'}: {ms:.3f} ms")
        if ms < best_ms:
            best, best_ms = eff, ms
    ctx.sync_status()
    ctx.set_tile_cap(best)
    _CACHE[key] = best
    del scratch
    return best
