"""Autotuner of the fused step's launch shape, with a persistent cache.

Two knobs, both in the context (the step's results do not depend on them, only its speed):

* the group capacity (particles per warp): the mixed path runs each cell on one CTA of 32 << k threads, k the
  smallest size class whose capacity (capacity << k particles) holds the cell, so the capacity sets the class
  thresholds, hence the threads per cell and the shared memory per CTA (resident CTAs per SM);
* the tile of the one-CTA kernel (particles staged in shared memory per cell), which serves the FP64 path and the
  cells above the largest group class.

Each candidate is timed over one fused step on a scratch copy of the velocities (the caller's state is untouched),
with CUDA events on the current stream, after one untimed step. The winner is cached per (device, library source,
precision, relativistic, cells, particles, largest cell) in memory and in a JSON file (``MCC_AUTOTUNE_CACHE``, default
``~/.cache/paper_2407_19151_gb300/autotune.json``), and applied to the context.
"""
from __future__ import annotations

import json
import os

import torch

from . import _binding as B
from ._build import source_hash

_CACHE: dict[str, dict] = {}
GROUP_CANDIDATES = (0, 128, 160, 192, 224, 256, 320, 384)       # 0: automatic (shared memory per SM / 16 warps)
TILE_CANDIDATES = (0, 128, 192, 256, 384, 512, 768, 1024, 1536, 2048)


def cache_path() -> str:
    return os.environ.get("MCC_AUTOTUNE_CACHE") or os.path.join(
        os.path.expanduser("~"), ".cache", "paper_2407_19151_gb300", "autotune.json")


def _load(path: str) -> dict:
    try:
        with open(path) as f:
            d = json.load(f)
        return d if isinstance(d, dict) else {}
    except (OSError, ValueError):
        return {}


def _store(path: str, key: str, value: dict) -> None:
    """Merge one entry into the cache file (write to a temporary file, then rename)."""
    try:
        os.makedirs(os.path.dirname(path) or ".", exist_ok=True)
        d = _load(path)
        d[key] = value
        tmp = f"{path}.tmp{os.getpid()}"
        with open(tmp, "w") as f:
            json.dump(d, f, indent=1, sort_keys=True)
        os.replace(tmp, path)
    except OSError:
        pass  # a read-only home only loses the persistence


def cache_key(device_name: str, sm_count: int, prec: str, relativistic: bool, n_cells: int, n_particles: int,
              max_cell: int, library: str) -> str:
    return "|".join(str(x) for x in (device_name, sm_count, library, prec, int(bool(relativistic)), n_cells,
                                     n_particles, max_cell))


def search(candidates, apply, time_one, verbose: bool = False, label: str = "") -> tuple[int, float]:
    """Apply each candidate, time it (time_one returns ms, or None if the candidate failed), keep the fastest;
    the winner is applied again at the end. Candidates that coincide (apply returns the same effective value) are
    timed once."""
    seen = set()
    best, best_ms = None, float("inf")
    for cand in candidates:
        eff = apply(cand)
        if eff in seen:
            continue
        seen.add(eff)
        ms = time_one()
        if verbose:
            print(f"autotune {label} {cand or 'auto'}: {ms if ms is None else round(ms, 3)} ms")
        if ms is not None and ms < best_ms:
            best, best_ms = cand, ms
    if best is None:
        best = candidates[0]
    apply(best)
    return best, best_ms


def autotune(vx, vy, vz, w, offsets, n_cells: int, n_species: int, species, lnL, params: B.Params, max_cell: int,
             interactions=None, persist: bool = True, verbose: bool = False) -> dict:
    """Pick and apply the group capacity (mixed path) and the one-CTA kernel's tile for this workload; returns
    {"group_cap", "tile_cap", "ms", "cached"} (0 = automatic)."""
    dev = vx.device
    ctx = B.context(dev)
    f32 = vx.dtype == torch.float32
    props = torch.cuda.get_device_properties(dev)
    key = cache_key(props.name, props.multi_processor_count, "f32" if f32 else "f64", params.relativistic, n_cells,
                    vx.numel(), max_cell, source_hash())
    path = cache_path()
    hit = _CACHE.get(key) or (_load(path).get(key) if persist else None)
    if hit:
        ctx.set_group_capacity(int(hit["group_cap"]))
        ctx.set_tile_cap(int(hit["tile_cap"]))
        _CACHE[key] = hit
        return dict(hit, cached=True)

    scratch = [x.clone() for x in (vx, vy, vz)]
    corr = torch.zeros(max(n_cells, 1), dtype=torch.int32, device=dev)
    fail = torch.zeros_like(corr)
    stream = torch.cuda.current_stream(dev)

    def time_one():
        try:
            B.mcc_step_fused(*scratch, w, offsets, n_cells, n_species, species, lnL, params, 1, max_cell,
                             interactions, corr, fail)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            B.mcc_step_fused(*scratch, w, offsets, n_cells, n_species, species, lnL, params, 1, max_cell,
                             interactions, corr, fail)
            e1.record(stream)
            torch.cuda.synchronize(dev)
        except B.MccError:
            return None
        return e0.elapsed_time(e1)

    rel = bool(params.relativistic)
    prec = B.F32_MIXED if f32 else B.F64

    def apply_group(cap):
        ctx.set_group_capacity(cap)
        return tuple(ctx.group_capacities(prec, rel))

    def apply_tile(cap):
        ctx.set_tile_cap(cap)
        return min(cap, max_cell) if cap else 0

    ctx.set_tile_cap(0)
    group, ms = (0, None)
    if f32:
        group, ms = search(GROUP_CANDIDATES, apply_group, time_one, verbose, "group capacity")
    tile = 0
    if not f32 or max_cell > ctx.group_capacities(prec, rel)[-1]:  # the one-CTA kernel runs some cells
        tile, ms = search(TILE_CANDIDATES, apply_tile, time_one, verbose, "tile")
    ctx.sync_status()
    del scratch
    out = {"group_cap": int(group), "tile_cap": int(tile), "ms": ms}
    _CACHE[key] = out
    if persist:
        _store(path, key, out)
    return dict(out, cached=False)
