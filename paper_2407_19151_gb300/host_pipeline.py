"""Collision steps on a state held in host memory, with the transfers overlapped with the compute.

Cells are independent within a step and across steps (the collision acts per cell; positions are frozen), so the
binned state splits into contiguous cell chunks. Chunk k is copied in on one stream, stepped ``n_steps`` times on a
second (one persistent kernel per step, random draws keyed by the global cell id, so the result equals the
unchunked run bit for bit), and copied out on a third, while chunk k + 1 is already being copied in. Device memory is
a ring of ``buffers`` chunk-sized slots; only the transfers and the stream ordering live here, every step runs in the
library's kernels (``mcc_step_fused``).
"""
from __future__ import annotations

import dataclasses

import numpy as np
import torch

from . import _binding as B
from .sharding import shard_cells, shard_view


def step_host(vx, vy, vz, w, offsets, n_cells: int, n_species: int, species, lnL, params: B.Params,
              n_steps: int = 1, max_cell: int | None = None, chunks: int = 4, buffers: int = 2, device=0,
              interactions=None):
    """Advance the host state (vx, vy, vz: pinned CPU tensors, float32 or float64; w: pinned float64) by n_steps
    in place. offsets: host int64 segment offsets. Returns the per-cell (corr_pairs, fail_count) as host arrays."""
    if getattr(params, "step_device", None) is not None:
        raise ValueError("step_host takes the step index from params.step (one call per step range)")
    dev = torch.device("cuda", device) if isinstance(device, int) else torch.device(device)
    off = np.asarray(offsets, dtype=np.int64)
    if max_cell is None:
        max_cell = int((off[n_species::n_species] - off[:-1:n_species]).max()) if n_cells else 0
    chunks = max(1, min(int(chunks), max(n_cells, 1)))
    ranges = [shard_cells(off, n_species, chunks, k) for k in range(chunks)]
    ranges = [r for r in ranges if r[1] > r[0]]
    views = [shard_view(off, n_species, c0, c1) for c0, c1 in ranges]
    cap_p = max((p1 - p0 for _, p0, p1 in views), default=0)
    cap_c = max((c1 - c0 for c0, c1 in ranges), default=0)
    nb = max(1, min(int(buffers), len(ranges)))
    vdt = vx.dtype
    slots = [dict(v=[torch.empty(max(cap_p, 1), dtype=vdt, device=dev) for _ in range(3)],
                  w=torch.empty(max(cap_p, 1), dtype=torch.float64, device=dev),
                  corr=torch.zeros(max(cap_c, 1), dtype=torch.int32, device=dev),
                  fail=torch.zeros(max(cap_c, 1), dtype=torch.int32, device=dev)) for _ in range(nb)]
    offs = [torch.from_numpy(local).to(dev) for local, _, _ in views]
    corr_h = torch.zeros(max(n_cells, 1), dtype=torch.int32).pin_memory()
    fail_h = torch.zeros(max(n_cells, 1), dtype=torch.int32).pin_memory()
    s_in, s_run, s_out = torch.cuda.Stream(dev), torch.cuda.Stream(dev), torch.cuda.Stream(dev)
    freed = [None] * nb
    for k, ((c0, c1), (_, p0, p1)) in enumerate(zip(ranges, views)):
        sl = slots[k % nb]
        n = p1 - p0
        with torch.cuda.stream(s_in):
            if freed[k % nb] is not None:
                s_in.wait_event(freed[k % nb])
            for dst, src in zip(sl["v"], (vx, vy, vz)):
                dst[:n].copy_(src[p0:p1], non_blocking=True)
            sl["w"][:n].copy_(w[p0:p1], non_blocking=True)
            loaded = torch.cuda.Event()
            loaded.record(s_in)
        with torch.cuda.stream(s_run):
            s_run.wait_event(loaded)
            sl["corr"].zero_()
            sl["fail"].zero_()
            p = dataclasses.replace(params, cell_base=int(params.cell_base) + c0)
            B.mcc_step_fused(*(x[:n] for x in sl["v"]), sl["w"][:n], offs[k], c1 - c0, n_species, species, lnL, p,
                             n_steps=n_steps, max_cell=max_cell, interactions=interactions, corr_pairs=sl["corr"],
                             fail_count=sl["fail"], stream=s_run)
            done = torch.cuda.Event()
            done.record(s_run)
        with torch.cuda.stream(s_out):
            s_out.wait_event(done)
            for dst, src in zip((vx, vy, vz), sl["v"]):
                dst[p0:p1].copy_(src[:n], non_blocking=True)
            corr_h[c0:c1].copy_(sl["corr"][: c1 - c0], non_blocking=True)
            fail_h[c0:c1].copy_(sl["fail"][: c1 - c0], non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(s_out)
            freed[k % nb] = ev
    for s in (s_in, s_run, s_out):
        s.synchronize()
    return corr_h[:n_cells].numpy(), fail_h[:n_cells].numpy()
