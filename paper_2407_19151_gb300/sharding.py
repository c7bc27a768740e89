"""Sharding of the collision step across GPUs. Cells are independent within a step (the collision acts per cell,
Sec. 2), so a problem splits into contiguous cell ranges with no exchange in the data path; every random draw is
keyed by the global cell id (``Params.cell_base``), so the union of the shards equals the unsharded run bit for
bit. The only collective is an optional all-reduce of per-species diagnostics."""
from __future__ import annotations

import numpy as np


def shard_cells(offsets, n_species: int, world: int, rank: int) -> tuple[int, int]:
    """Contiguous cell range [c0, c1) of `rank`, balanced by particle count (prefix sums over cells)."""
    off = np.asarray(offsets, dtype=np.int64)
    cell_start = off[::n_species]            # n_cells + 1 particle offsets at cell boundaries
    n_cells = len(cell_start) - 1
    total = int(cell_start[-1])
    bounds = [0]
    for r in range(1, world):
        target = total * r / world
        bounds.append(int(np.searchsorted(cell_start, target, side="left")))
    bounds.append(n_cells)
    bounds = np.maximum.accumulate(np.clip(bounds, 0, n_cells))
    return int(bounds[rank]), int(bounds[rank + 1])


def shard_view(offsets, n_species: int, c0: int, c1: int):
    """Rebased segment offsets of cells [c0, c1) and their particle range [p0, p1) in the global arrays."""
    off = np.asarray(offsets, dtype=np.int64)
    local = off[c0 * n_species: c1 * n_species + 1]
    p0, p1 = int(local[0]), int(local[-1])
    return local - p0, p0, p1


def species_moments(vx, vy, vz, w, offsets, n_cells: int, n_species: int, m):
    """Per-species totals (sum w, sum m w v (3), sum 1/2 m w v^2) of a binned state, for the diagnostics
    all-reduce; returns an (n_species, 5) float64 array."""
    off = np.asarray(offsets, dtype=np.int64)
    sp = np.repeat(np.tile(np.arange(n_species), n_cells), np.diff(off))
    v = np.stack([np.asarray(vx, np.float64), np.asarray(vy, np.float64), np.asarray(vz, np.float64)], axis=1)
    w = np.asarray(w, np.float64)
    out = np.zeros((n_species, 5))
    mw = np.asarray(m, np.float64)[sp] * w
    np.add.at(out[:, 0], sp, w)
    for d in range(3):
        np.add.at(out[:, 1 + d], sp, mw * v[:, d])
    np.add.at(out[:, 4], sp, 0.5 * mw * (v ** 2).sum(1))
    return out
