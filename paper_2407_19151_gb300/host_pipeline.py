"""Collision steps on a state held in host memory, with the transfers overlapped with the compute.

Cells are independent within a step and across steps (the collision acts per cell; positions are frozen), so the
binned state splits into contiguous cell chunks. Chunk k is copied in on one stream, stepped ``n_steps`` times on a
second (one mcc_step_fused call, random draws keyed by the global cell id, so the result equals the unchunked run bit
for bit), and copied out on a third, while chunk k + 1 is already being copied in. With ``round_trips`` > 1 the state
makes that many round trips through host memory: chunk k of round trip t + 1 is copied in as soon as its copy out of
round trip t has landed, so the pipeline does not drain between round trips. Device memory is a ring of ``buffers``
chunk-sized slots; only the transfers and the stream ordering live here, every step runs in the library's kernels.
"""
from __future__ import annotations

import dataclasses

import numpy as np
import torch

from . import _binding as B
from .sharding import shard_cells, shard_view


def step_host(vx, vy, vz, w, offsets, n_cells: int, n_species: int, species, lnL, params: B.Params,
              n_steps: int = 1, max_cell: int | None = None, chunks: int = 4, buffers: int = 2, device=0,
              interactions=None, round_trips: int = 1):
    """Advance the host state (vx, vy, vz: pinned CPU tensors, float32 or float64; w: pinned float64) in place by
    round_trips x n_steps steps: every round trip copies each chunk in, runs n_steps steps on it (step indices
    params.step + t n_steps + 0 .. n_steps - 1 in round trip t) and copies it back. offsets: host int64 segment
    offsets. Returns the per-cell (corr_pairs, fail_count), accumulated over all steps, as host arrays."""
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
    nb = max(1, min(int(buffers), len(ranges)))
    vdt = vx.dtype
    slots = [dict(v=[torch.empty(max(cap_p, 1), dtype=vdt, device=dev) for _ in range(3)],
                  w=torch.empty(max(cap_p, 1), dtype=torch.float64, device=dev)) for _ in range(nb)]
    offs = [torch.from_numpy(local).to(dev) for local, _, _ in views]
    # per-chunk counters on the device, accumulated over every step, copied out once at the end
    corr = [torch.zeros(max(c1 - c0, 1), dtype=torch.int32, device=dev) for c0, c1 in ranges]
    fail = [torch.zeros(max(c1 - c0, 1), dtype=torch.int32, device=dev) for c0, c1 in ranges]
    s_in, s_run, s_out = torch.cuda.Stream(dev), torch.cuda.Stream(dev), torch.cuda.Stream(dev)
    freed = [None] * nb                  # slot free again (its chunk copied out)
    landed = [None] * len(ranges)        # chunk's previous round trip back in host memory
    job = 0
    for t in range(max(1, int(round_trips))):
        for k, ((c0, c1), (_, p0, p1)) in enumerate(zip(ranges, views)):
            slot = job % nb
            job += 1
            sl = slots[slot]
            n = p1 - p0
            with torch.cuda.stream(s_in):
                if freed[slot] is not None:
                    s_in.wait_event(freed[slot])
                if landed[k] is not None:
                    s_in.wait_event(landed[k])
                for dst, src in zip(sl["v"], (vx, vy, vz)):
                    dst[:n].copy_(src[p0:p1], non_blocking=True)
                sl["w"][:n].copy_(w[p0:p1], non_blocking=True)
                loaded = torch.cuda.Event()
                loaded.record(s_in)
            with torch.cuda.stream(s_run):
                s_run.wait_event(loaded)
                p = dataclasses.replace(params, cell_base=int(params.cell_base) + c0,
                                        step=int(params.step) + t * int(n_steps))
                B.mcc_step_fused(*(x[:n] for x in sl["v"]), sl["w"][:n], offs[k], c1 - c0, n_species, species, lnL,
                                 p, n_steps=n_steps, max_cell=max_cell, interactions=interactions,
                                 corr_pairs=corr[k], fail_count=fail[k], stream=s_run)
                done = torch.cuda.Event()
                done.record(s_run)
            with torch.cuda.stream(s_out):
                s_out.wait_event(done)
                for dst, src in zip((vx, vy, vz), sl["v"]):
                    dst[p0:p1].copy_(src[:n], non_blocking=True)
                ev = torch.cuda.Event()
                ev.record(s_out)
                freed[slot] = ev
                landed[k] = ev
    corr_h = torch.zeros(max(n_cells, 1), dtype=torch.int32)
    fail_h = torch.zeros(max(n_cells, 1), dtype=torch.int32)
    for s in (s_in, s_run, s_out):
        s.synchronize()
    for (c0, c1), cr, fl in zip(ranges, corr, fail):
        corr_h[c0:c1] = cr[: c1 - c0].cpu()
        fail_h[c0:c1] = fl[: c1 - c0].cpu()
    return corr_h[:n_cells].numpy(), fail_h[:n_cells].numpy()
