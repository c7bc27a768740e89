"""PIC coupling: collision steps on particles that move between them.

A particle-in-cell code advances positions (the Vlasov part of Eq. Boltzmann, Sec. 2) between applications of the
collision operator, so the cell sort is no longer a one-time cost: after every push the particles are re-binned
before the next collision step. One step here is

    push (mcc_push: x += v dt, periodic box, new cell ids)
    -> cell sort (mcc_bin: stable by cell and species; or mcc_bin_weighted: each segment by descending weight, the
       layout in which the step skips its per-visit weight sort)
    -> one gather pass of every particle array through the permutation (mcc_gather_n)
    -> collision step (mcc_step_fused)

with the acceleration of the push set to zero (no field solve: the paper gives none). Every stage is a kernel of
the CUDA library; this module holds the buffers and orders the calls.
"""
from __future__ import annotations

import dataclasses

import torch

from . import _binding as B


class PicLoop:
    """Particle state (positions, velocities, weights, species ids, all binned) with spare buffers for the re-bin.

    x, y, z, vx, vy, vz share one dtype (float64: FP64 step; float32: mixed step); w float64; species int32;
    offsets int64 of the current binning. The arrays are replaced (not modified in place) by each step's gather.
    """

    def __init__(self, x, y, z, vx, vy, vz, w, species, offsets, n_cells: int, n_species: int, grid,
                 species_params, lnL, params: B.Params, dt_push: float, interactions=None, order: str = "stable"):
        if order not in ("stable", "weight"):
            raise ValueError("order is 'stable' or 'weight'")
        self.order = order
        self.arrays = [x, y, z, vx, vy, vz, w, species]
        self.spare = [torch.empty_like(a) for a in self.arrays]
        self.cell = torch.empty(x.numel(), dtype=torch.int32, device=x.device)
        self.offsets = offsets
        self.n_cells, self.n_species = int(n_cells), int(n_species)
        self.grid = grid
        self.sp = list(species_params)
        self.lnL = lnL
        self.params = params
        self.dt_push = float(dt_push)
        self.inter = interactions
        self.t = 0

    @property
    def state(self):
        """(x, y, z, vx, vy, vz, w, species) of the current binning."""
        return tuple(self.arrays)

    def push_and_rebin(self, stream=None):
        x, y, z, vx, vy, vz, w, sp = self.arrays
        B.mcc_push(x, y, z, vx, vy, vz, self.grid, self.dt_push, self.params.relativistic, self.params.c,
                   cell=self.cell, stream=stream)
        if self.order == "weight":
            perm, self.offsets = B.mcc_bin_weighted(self.cell, sp, w, self.n_cells, self.n_species, stream=stream)
        else:
            perm, self.offsets = B.mcc_bin(self.cell, sp, self.n_cells, self.n_species, stream=stream)
        B.mcc_gather_n(self.arrays, perm, outs=self.spare, stream=stream)
        self.arrays, self.spare = self.spare, self.arrays

    def step(self, n_steps: int = 1, max_cell: int | None = None, stream=None):
        """n_steps of push, re-bin and collision; returns the per-cell energy-pair and failure counts summed over
        the steps (cells are re-populated between steps, so these are per cell id). max_cell: a bound on particles
        per cell after any re-bin (None: read from the offsets each step, one host synchronisation per step)."""
        dev = self.arrays[0].device
        corr = torch.zeros(max(self.n_cells, 1), dtype=torch.int32, device=dev)
        fail = torch.zeros(max(self.n_cells, 1), dtype=torch.int32, device=dev)
        for _ in range(int(n_steps)):
            self.push_and_rebin(stream)
            vx, vy, vz, w = self.arrays[3:7]
            p = dataclasses.replace(self.params, step=self.params.step + self.t)
            B.mcc_step_fused(vx, vy, vz, w, self.offsets, self.n_cells, self.n_species, self.sp, self.lnL, p,
                             n_steps=1, max_cell=max_cell, interactions=self.inter, corr_pairs=corr,
                             fail_count=fail, stream=stream)
            self.t += 1
        return corr[:self.n_cells], fail[:self.n_cells]
