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


class CudaShard:
    """Device side of one rank's shard: the particles of cells [c0, c1) on this rank's GPU, stepped by
    mcc_step_fused with cell_base = c0 and summarised by mcc_species_moments."""

    def __init__(self, device=None):
        import torch
        self.device = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)

    def load(self, vx, vy, vz, w, view):
        """This rank's slice of the global host arrays (p0:p1 of view) as device tensors, with the rebased
        offsets."""
        import torch
        local, p0, p1, _, _ = view
        to = lambda a: torch.from_numpy(np.ascontiguousarray(a[p0:p1])).to(self.device)  # noqa: E731
        return {"v": [to(vx), to(vy), to(vz)], "w": to(w), "offsets": torch.from_numpy(local).to(self.device)}

    def step(self, st, n_cells, S, species, lnL, params, n_steps, max_cell, fail):
        from . import _binding as B
        B.mcc_step_fused(*st["v"], st["w"], st["offsets"], n_cells, S, species, lnL, params, n_steps=n_steps,
                         max_cell=max_cell, fail_count=fail)

    def zeros(self, n):
        import torch
        return torch.zeros(max(n, 1), dtype=torch.int32, device=self.device)

    def moments(self, st, n_cells, S, species, params, fail):
        from . import _binding as B
        return B.mcc_species_moments(*st["v"], st["w"], st["offsets"], n_cells, S, species, params.relativistic,
                                     params.c, fail)

    def velocities(self, st):
        return np.stack([x.double().cpu().numpy() for x in st["v"]], axis=1)


class ShardedStep:
    """The collision step of one problem split over the ranks of a torch.distributed process group, one GPU per
    rank. Rank r owns the contiguous, particle-balanced cell range [c0, c1) of the global segment offsets
    (shard_cells) and holds only those particles; step() runs the fused step on them with cell_base = c0, so every
    draw is keyed by the global cell id and the union of the shards equals the unsharded run bit for bit. The data
    path exchanges nothing (the collision acts per cell, Sec. 2); the one collective is the all-reduce (sum) of the
    per-species diagnostics (sum w, momentum, kinetic energy, count per species, and the failed corrections), once
    per call of step(). Without an initialised process group it runs the whole problem as one rank.

        sh = ShardedStep(offsets, n_cells, S, species, lnL, params)   # host int64 global offsets
        sh.load(vx, vy, vz, w)                                         # global host arrays; keeps this rank's part
        diag = sh.step(n_steps)                                        # (S, 6) sums over all ranks, failures

    `backend` is the device side (CudaShard by default); it is a parameter so that the host logic can be exercised
    on CPU ranks with another implementation of the same five calls."""

    def __init__(self, offsets, n_cells: int, n_species: int, species, lnL, params, group=None, backend=None,
                 max_cell: int | None = None, cell_range: tuple[int, int] | None = None):
        import dataclasses

        import torch.distributed as dist
        self.dist = dist if dist.is_available() and dist.is_initialized() else None
        self.group = group
        self.rank = self.dist.get_rank(group) if self.dist else 0
        self.world = self.dist.get_world_size(group) if self.dist else 1
        off = np.asarray(offsets, dtype=np.int64)
        self.S = int(n_species)
        self.c0, self.c1 = cell_range if cell_range is not None else shard_cells(off, self.S, self.world, self.rank)
        local, self.p0, self.p1 = shard_view(off, self.S, self.c0, self.c1)
        self.view = (local, self.p0, self.p1, self.c0, self.c1)
        self.n_cells = self.c1 - self.c0
        counts = off[self.S::self.S] - off[:-1:self.S]
        self.max_cell = int(counts.max()) if max_cell is None and len(counts) else int(max_cell or 0)
        self.species = list(species)
        self.lnL = lnL
        self.params = dataclasses.replace(params, cell_base=int(params.cell_base) + self.c0)
        self.backend = backend if backend is not None else CudaShard()
        self.state = None
        self.fail = None

    def load(self, vx, vy, vz, w, local: bool = False):
        """Take this rank's particles: from the global host arrays (binned by the global offsets), or, with
        local=True, arrays that hold exactly this rank's particles."""
        if local:
            n = self.p1 - self.p0
            if len(vx) != n:
                raise ValueError(f"this rank holds {n} particles, got {len(vx)}")
            view = (self.view[0], 0, n, self.c0, self.c1)
            self.state = self.backend.load(vx, vy, vz, w, view)
        else:
            self.state = self.backend.load(vx, vy, vz, w, self.view)
        self.fail = self.backend.zeros(self.n_cells)
        return self

    def advance(self, n_steps: int = 1):
        """n_steps collision steps of this rank's cells (no collective)."""
        if self.state is None:
            raise RuntimeError("load() the particles first")
        if self.n_cells > 0 and n_steps > 0:
            self.backend.step(self.state, self.n_cells, self.S, self.species, self.lnL, self.params, n_steps,
                              self.max_cell, self.fail)
        self.params.step = int(self.params.step) + n_steps

    def step(self, n_steps: int = 1):
        """n_steps collision steps of this rank's cells, then the diagnostics summed over the ranks: an (S, 6)
        array (sum w, sum m w v (3), kinetic energy, count) and the failed corrections accumulated since load()."""
        self.advance(n_steps)
        return self.diagnostics()

    def diagnostics(self):
        """The per-species diagnostics of the current state summed over the ranks (one all-reduce)."""
        d = self.backend.moments(self.state, self.n_cells, self.S, self.species, self.params, self.fail)
        if self.dist is not None and self.world > 1:
            self.dist.all_reduce(d, group=self.group)
        d = d.cpu().numpy() if hasattr(d, "cpu") else np.asarray(d)
        return d[:6 * self.S].reshape(self.S, 6), int(round(float(d[6 * self.S])))

    def velocities(self):
        """This rank's velocities (its particles p0:p1 of the global arrays), on the host."""
        return self.backend.velocities(self.state)
