"""Benchmark of the fused collision step on the three-species plasma (2^18 cells, log-normal counts with mean 512,
about 1.34e8 particles, N97, float velocities with double weights and float-float moment sums). Each (cell, species)
segment is stored by descending weight, the order mcc_bin_weighted produces (``--layout generated`` keeps the
generated order, in which every cell visit also sorts its species by weight).

One step = one pass of the whole collision step over every cell and interaction (pairing, scatter, momentum and
energy correction), one persistent kernel launch. K steps are captured in one CUDA graph and timed with CUDA events
on the launching stream; the state (4.3 GB read + written per step) is far larger than L2, so no flush is needed.

Prints one JSON line: collision pairs/s (scatter pairs of all interactions; a triplet counts three) with the HBM
roofline of the step kernel, the end-to-end figure through host buffers, the plain FP64 GPU step on the same
workload, and the oracle timed on the host cores on a bounded sample of cells.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "collision pairs/sec"
UNIT = "pairs/s"
BYTES_PER_PARTICLE = {"f32": 32, "f64": 56}  # read v (12|24) + w (8), write v (12|24)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cells", type=int, default=1 << 18, help="cells of the three-species workload")
    ap.add_argument("--fp64-steps", type=int, default=3)
    ap.add_argument("--group-cap", type=int, default=None,
                    help="group capacity, particles per warp (0: automatic); default: the autotuner's choice")
    ap.add_argument("--tile-cap", type=int, default=None,
                    help="tile of the one-CTA kernel (0: automatic); default: the autotuner's choice")
    ap.add_argument("--layout", default="weight_ordered", choices=["weight_ordered", "generated"],
                    help="particle order within each (cell, species) segment: by descending weight, as mcc_bin_weighted "
                         "stores it, or as generated")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--e2e-chunks", type=int, default=8, help="cell chunks of the host-buffer pipeline")
    ap.add_argument("--e2e-buffers", type=int, default=3, help="device chunk slots of the host-buffer pipeline")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--no-bin", action="store_true")
    ap.add_argument("--no-configs", action="store_true", help="skip the other workloads' step times")
    ap.add_argument("--no-pic", action="store_true", help="skip the PIC-coupling (push, re-bin, step) timing")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


DOMINANT_KERNEL_SOURCES = ("mcc_group.cuh", "mcc_group_f32.cu", "mcc_device.cuh", "mcc_kernels.h")


def kernel_source_hash() -> str:
    """Hash of the sources the mixed-path group kernels are compiled from (the committed ncu record is valid only
    for the kernel source it was taken on)."""
    from paper_2407_19151_gb300 import _build
    h = hashlib.sha256()
    for f in DOMINANT_KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_2407_19151_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    h.update(" ".join(_build.UNIT_FLAGS.get("mcc_group_f32.cu", [])).encode())  # the unit's compile flags
    return h.hexdigest()[:16]


def ncu_entry(workload: str):
    """The committed ncu summary of the step kernel (DRAM bytes per launch, issue-slot use), if it was taken on this
    kernel source; otherwise None."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            d = json.load(f)
        e = d.get(workload)
        if e and e.get("kernel_source") == kernel_source_hash():
            return e
    except Exception:
        pass
    return None


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        out_dir = os.environ.get("MCC_BENCH_OUT") or os.path.join(tempfile.gettempdir(), "mcc_bench")
        self.path = os.path.join(out_dir, f"clocks_bench_{index}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}",
                 "--query-gpu=clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
                 "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
                 "clocks_event_reasons.sw_power_cap",
                 "--format=csv,noheader,nounits", "-lms", "100"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        try:
            rows = [r.split(",") for r in open(self.path).read().strip().splitlines() if r.strip()]
            if not rows:
                raise ValueError("no clock samples")
            sm = [float(r[0]) for r in rows]
            mx = [float(r[1]) for r in rows]
            names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
            reasons = sorted({names[k] for r in rows for k in range(4) if r[3 + k].strip().lower() == "active"})
            return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "reasons": reasons,
                    "samples": len(rows)}
        except Exception:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}


def make_workload(cells: int, rank: int, precision: str, layout: str = "weight_ordered"):
    from paper_2407_19151_gb300 import workloads as W
    wl = W.three_species(n_cells=cells, data_seed=1239 + 1000 * rank, precision=precision)
    return wl.weight_ordered() if layout == "weight_ordered" else wl


PRECISION = ("f32 velocities and kinematics, f64 weights; float-float (about 2^-44) sums, coefficients and "
             "on-chip cell state")


def bench_config(wl, layout: str, world: int) -> dict:
    """The workload description both arms print (same keys, same values)."""
    return {"workload": "three_species", "n_cells": wl.n_cells, "n_particles": wl.n, "species": wl.n_species,
            "interactions": len(wl.interactions()), "pairs_per_step": wl.pairs_per_step(), "method": "N97",
            "max_cell": int(wl.counts.sum(axis=1).max()),
            "layout": layout + (" (segments by descending weight, the mcc_bin_weighted order)"
                                if layout == "weight_ordered" else ""),
            "l2": f"no flush: {32 * wl.n / 1e9:.2g} GB of state read and written per step (129 MB L2)",
            "parallelism": (f"cells: one problem in {world} shards (ShardedStep), diagnostics all-reduce" if world > 1
                            else "cells: one problem on one GPU")}


def cpu_baseline(wl, budget_s: float = 15.0, one_thread: bool = False):
    """The oracle as it stands on the host cores (OpenMP over cells), on the first cells of the same workload:
    grows the sample until a run takes a few seconds, then reports pairs/s."""
    import oracle as O
    cores = os.cpu_count() or 1
    os.environ.setdefault("OMP_NUM_THREADS", str(cores))
    k = 64
    spent = 0.0
    best = None
    while True:
        sub = wl.subset(k)
        st = O.State(sub.vx.astype(np.float64), sub.vy.astype(np.float64), sub.vz.astype(np.float64), sub.w,
                     sub.offsets, sub.n_cells, sub.n_species)
        p = O.Params(method=sub.method, dt=sub.dt, dV=sub.dV, eps0=sub.eps0, c=sub.c, fE=sub.fE, seed=sub.seed)
        t0 = time.perf_counter()
        O.step(st, sub.q, sub.m, sub.lnL, p, n_steps=1)
        dt = time.perf_counter() - t0
        spent += dt
        best = (sub.pairs_per_step() / dt, k, dt)
        if dt > budget_s / 3 or spent > budget_s or k >= wl.n_cells:
            break
        k = min(wl.n_cells, int(k * max(2.0, (budget_s / 3) / max(dt, 1e-3))))
    out = {"value": best[0], "unit": UNIT, "cores": int(os.environ["OMP_NUM_THREADS"]), "kind": "oracle",
           "sample": f"one step of the first {best[1]} cells ({best[2]:.1f} s, FP64 C oracle, OpenMP over cells)"}
    if one_thread:
        # the same oracle on one host thread, on the first 1024 cells
        k = min(1024, wl.n_cells)
        sub = wl.subset(k)
        st = O.State(sub.vx.astype(np.float64), sub.vy.astype(np.float64), sub.vz.astype(np.float64), sub.w,
                     sub.offsets, sub.n_cells, sub.n_species)
        p = O.Params(method=sub.method, dt=sub.dt, dV=sub.dV, eps0=sub.eps0, c=sub.c, fE=sub.fE, seed=sub.seed)
        O.set_threads(1)
        t0 = time.perf_counter()
        O.step(st, sub.q, sub.m, sub.lnL, p, n_steps=1)
        dt = time.perf_counter() - t0
        O.set_threads(cores)
        out["one_thread"] = {"value": sub.pairs_per_step() / dt, "unit": UNIT,
                             "sample": f"one step of the first {k} cells ({dt:.1f} s, one thread)"}
    return out


def run_reference(args):
    rank, _, _ = dist_env()
    if rank != 0:
        return
    wl = make_workload(args.cells, 0, "f32", args.layout)
    cb = cpu_baseline(wl, budget_s=max(5.0, 60.0 / max(1, args.steps + args.warmup)))
    line = {"impl": "reference", "metric": METRIC, "value": cb["value"], "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": bench_config(wl, args.layout, args.gpus),
            "cpu_baseline": cb, "e2e": {"value": cb["value"], "unit": UNIT, "h2d_bytes_per_step": 0,
                                        "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def configs_measure(dev, hbm):
    """Step time of the other synthetic workloads (the paper's test plasmas at GPU sizes): isotropisation (FP64),
    equilibration (mixed, TA77 and N97), relativistic beam (mixed). Fused steps, CUDA events, after two warm-up
    steps; pairs/s and the HBM fraction of their algorithmic bytes."""
    import torch

    import paper_2407_19151_gb300 as mcc
    from paper_2407_19151_gb300 import workloads as W
    cases = [("isotropisation", W.isotropisation(), "f64"),
             ("equilibration_ta77", W.equilibration(method=W.TA77), "f32"),
             ("equilibration_n97", W.equilibration(method=W.N97), "f32"),
             ("relativistic_beam", W.relativistic_beam(), "f32")]
    out = {}
    stream = torch.cuda.current_stream(dev)
    for name, wl, prec in cases:
        dt_ = torch.float64 if prec == "f64" else torch.float32
        v = [torch.tensor(np.asarray(x), dtype=dt_, device=dev) for x in (wl.vx, wl.vy, wl.vz)]
        w = torch.from_numpy(wl.w).to(dev)
        off = torch.from_numpy(wl.offsets).to(dev)
        sp = list(zip(wl.q.tolist(), wl.m.tolist()))
        mc = int(wl.counts.sum(axis=1).max())
        p = mcc.Params(method=wl.method, relativistic=wl.relativistic, dt=wl.dt, fE=wl.fE, c=wl.c, seed=wl.seed)
        mcc.mcc_step_fused(*v, w, off, wl.n_cells, wl.n_species, sp, wl.lnL, p, n_steps=2, max_cell=mc)
        torch.cuda.synchronize(dev)
        k = 10
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        p.step = 2
        e0.record(stream)
        mcc.mcc_step_fused(*v, w, off, wl.n_cells, wl.n_species, sp, wl.lnL, p, n_steps=k, max_cell=mc)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        mcc.sync_status(dev.index or 0)
        ms = e0.elapsed_time(e1) / k
        out[name] = {"precision": prec, "n_cells": wl.n_cells, "n_particles": wl.n, "ms_per_step": ms,
                     "pairs_per_s": wl.pairs_per_step() / (ms * 1e-3),
                     "hbm_frac": BYTES_PER_PARTICLE[prec] * wl.n / (ms * 1e-3) / 1e9 / hbm}
    return out


def bin_measure(wl, dev):
    """One-time cell sort of the same particles from a shuffled order (row a1, reported apart from the step):
    mcc_bin (stable by cell and species), mcc_bin_weighted (segments by descending weight) and the gather of
    vx, vy, vz, w through the permutation; CUDA events, after one untimed call each."""
    import torch

    import paper_2407_19151_gb300 as mcc
    rng = np.random.default_rng(7)
    order = rng.permutation(wl.n)
    cell = torch.from_numpy(wl.cell_of_particles()[order]).to(dev)
    species = torch.from_numpy(wl.species_of_particles()[order]).to(dev)
    w = torch.from_numpy(wl.w[order]).to(dev)
    v = [torch.from_numpy(np.ascontiguousarray(x[order])).to(dev) for x in (wl.vx, wl.vy, wl.vz)]
    stream = torch.cuda.current_stream(dev)
    res = {}
    for name, fn in (("bin", lambda: mcc.mcc_bin(cell, species, wl.n_cells, wl.n_species)),
                     ("bin_weighted", lambda: mcc.mcc_bin_weighted(cell, species, w, wl.n_cells, wl.n_species))):
        fn()
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        perm, _ = fn()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        res[name + "_ms"] = e0.elapsed_time(e1)
    mcc.sync_status(dev.index or 0)
    for x in (*v, w):
        mcc.mcc_gather(x, perm)
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for x in (*v, w):
        mcc.mcc_gather(x, perm)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    res["gather_ms"] = e0.elapsed_time(e1)
    res["particles"] = wl.n
    res["note"] = "one-time cost (positions frozen in the step); the step itself reads the binned arrays"
    return res


def pic_measure(wl, dev, hbm, steps: int = 4):
    """PIC coupling on the same particles (row f3): positions in 64^3 unit cells (periodic), and per step the
    free-streaming push (drift Courant number 0.25 for the electrons' thermal speed), the re-bin (stable, or with
    segments by descending weight), one gather pass of the eight particle arrays, and the collision step. Each phase
    timed with CUDA events on the stream, after one untimed step; the re-bin is now a per-step cost."""
    import dataclasses

    import torch

    import paper_2407_19151_gb300 as mcc
    from paper_2407_19151_gb300 import workloads as W
    C, S = wl.n_cells, wl.n_species
    grid, x, y, z, dt_push = W.pic_setup(wl, cfl=0.25)
    sp = wl.species_of_particles()
    species = list(zip(wl.q.tolist(), wl.m.tolist()))
    stream = torch.cuda.current_stream(dev)
    out = {"grid": list(grid[0]), "cfl": 0.25, "dt_push": dt_push, "particles": wl.n}
    for order in ("weight", "stable"):
        to = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)  # noqa: E731
        arrays = [to(x), to(y), to(z), to(wl.vx), to(wl.vy), to(wl.vz), to(wl.w), to(sp)]
        spare = [torch.empty_like(a) for a in arrays]
        cell = torch.empty(wl.n, dtype=torch.int32, device=dev)
        off = torch.from_numpy(wl.offsets).to(dev)
        p = mcc.Params(method=wl.method, dt=wl.dt, fE=wl.fE, seed=wl.seed, step=5000)
        tot = {"push": 0.0, "bin": 0.0, "gather": 0.0, "step": 0.0}
        moved = 0.0
        pairs = 0
        for k in range(steps + 1):
            before = torch.repeat_interleave(torch.arange(C, device=dev, dtype=torch.int32),
                                             off[S::S] - off[:-1:S], output_size=wl.n)
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(6)]
            ev[0].record(stream)
            mcc.mcc_push(*arrays[:6], grid, dt_push, cell=cell)
            ev[1].record(stream)
            if order == "weight":
                perm, off = mcc.mcc_bin_weighted(cell, arrays[7], arrays[6], C, S)
            else:
                perm, off = mcc.mcc_bin(cell, arrays[7], C, S)
            ev[2].record(stream)
            mcc.mcc_gather_n(arrays, perm, outs=spare)
            ev[3].record(stream)
            arrays, spare = spare, arrays
            moved = float((cell != before).float().mean().item())
            counts = (off[1:] - off[:-1]).view(C, S).cpu().numpy()
            mc = int(counts.sum(axis=1).max())
            ev[4].record(stream)
            mcc.mcc_step_fused(*arrays[3:7], off, C, S, species, wl.lnL, dataclasses.replace(p, step=5000 + k),
                               n_steps=1, max_cell=mc)
            ev[5].record(stream)
            torch.cuda.synchronize(dev)
            if k > 0:
                for name, a, b in (("push", 0, 1), ("bin", 1, 2), ("gather", 2, 3), ("step", 4, 5)):
                    tot[name] += ev[a].elapsed_time(ev[b]) / steps
                pairs += dataclasses.replace(wl, counts=counts).pairs_per_step() / steps
        mcc.sync_status(dev.index or 0)
        ms = sum(tot.values())
        out[order] = {"ms_per_step": ms, "pairs_per_s": pairs / (ms * 1e-3),
                      **{f"{k}_ms": v for k, v in tot.items()}, "moved_fraction": moved,
                      "push_hbm_frac": 40 * wl.n / (tot["push"] * 1e-3) / 1e9 / hbm,
                      "gather_hbm_frac": 76 * wl.n / (tot["gather"] * 1e-3) / 1e9 / hbm}
        del arrays, spare, cell, perm, off
    out["note"] = ("push 40 B and gather 76 B of algorithmic traffic per particle (float positions and velocities); "
                   "'weight': re-bin with segments by descending weight (the step skips its weight sort); "
                   "'stable': plain stable re-bin")
    return out


def adjoint_measure(dev):
    """Differentiable step (1024 cells x 512 particles, two species of mass ratio 1836, FP64, N97): 50 steps, gradient
    of the final per-species temperatures and drifts with respect to the initial velocities, weights and Coulomb
    logarithms, once with a checkpoint every 10 steps and once with recorded tapes. Forward and backward timed
    separately with CUDA events."""
    import torch

    import paper_2407_19151_gb300 as mcc
    from paper_2407_19151_gb300 import workloads as W
    wl = W.differentiable(n_cells=1024, per_species=256)
    n_steps, every = 50, 10
    v = [torch.tensor(x, dtype=torch.float64, device=dev, requires_grad=True) for x in (wl.vx, wl.vy, wl.vz)]
    w = torch.tensor(wl.w, dtype=torch.float64, device=dev, requires_grad=True)
    L = torch.tensor(wl.lnL, dtype=torch.float64, requires_grad=True)
    off = torch.from_numpy(wl.offsets).to(dev)
    sp_of = torch.from_numpy(wl.species_of_particles()).to(dev).long()
    species = list(zip(wl.q.tolist(), wl.m.tolist()))
    params = mcc.Params(method=wl.method, dt=wl.dt, fE=wl.fE, seed=wl.seed, step=0)

    def temps_drifts(out):
        loss = 0.0
        for s in range(wl.n_species):
            sel = sp_of == s
            ws = w[sel]
            V = [torch.sum(ws * x[sel]) / torch.sum(ws) for x in out]
            T = sum(torch.sum(ws * (x[sel] - Vd) ** 2) for x, Vd in zip(out, V)) * wl.m[s] / (3 * torch.sum(ws))
            loss = loss + T + sum(V)
        return loss

    stream = torch.cuda.current_stream(dev)
    pairs = wl.pairs_per_step() * n_steps
    res = {"workload": "differentiable, 1024 cells x 512, two species, FP64, N97", "steps": n_steps}
    for mode, tape in (("checkpoint", False), ("tape", True)):
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        out = mcc.collision_steps(*v, w, L, off, wl.n_cells, wl.n_species, species, params, 2, checkpoint_every=every,
                                  tape=tape)
        temps_drifts(out).backward()  # warm-up (library load, workspaces)
        for x in (*v, w, L):
            x.grad = None
        torch.cuda.synchronize(dev)
        ev[0].record(stream)
        out = mcc.collision_steps(*v, w, L, off, wl.n_cells, wl.n_species, species, params, n_steps,
                                  checkpoint_every=every, tape=tape)
        loss = temps_drifts(out)
        ev[1].record(stream)
        loss.backward()
        ev[2].record(stream)
        torch.cuda.synchronize(dev)
        f_ms, b_ms = ev[0].elapsed_time(ev[1]), ev[1].elapsed_time(ev[2])
        res[mode] = {"forward_ms": f_ms, "backward_ms": b_ms, "backward_over_forward": b_ms / f_ms,
                     "pairs_per_s_forward_backward": pairs / ((f_ms + b_ms) * 1e-3),
                     "grad_norms": {"v": float(sum(x.grad.norm() ** 2 for x in v) ** 0.5),
                                    "w": float(w.grad.norm()), "lnL": float(L.grad.norm())}}
        for x in (*v, w, L):
            x.grad = None
        del out, loss
    res["checkpoint"]["checkpoint_every"] = every
    res["tape"]["tape_bytes"] = mcc.adjoint_tape_bytes(dev, wl.n_cells, int(wl.counts.sum(1).max()),
                                                       params.max_corr_passes) * n_steps * 3
    return res


CLASS_KERNELS = [f"group_kernel<false, {32 << k}>" for k in range(5)] + ["cell_kernel<float, 0, 0>"]


def class_table(wl, caps, class_ms, hbm):
    """Per size class (threads per cell 32 << k; last: the one-CTA kernel of the cells above every class): cells,
    particles, mean launch time, and the HBM rate of its 32 algorithmic bytes per particle."""
    n = wl.counts.sum(axis=1)
    cls = np.searchsorted(np.asarray(caps), n, side="left")  # smallest class whose capacity holds the cell
    rows = []
    for k in range(len(caps) + 1):
        sel = cls == k
        parts = int(n[sel].sum())
        ms = float(class_ms[k])
        gbs = BYTES_PER_PARTICLE["f32"] * parts / (ms * 1e-3) / 1e9 if ms > 0 and parts else 0.0
        rows.append({"kernel": CLASS_KERNELS[k], "capacity": int(caps[k]) if k < len(caps) else None,
                     "cells": int(sel.sum()), "particles": parts, "ms": ms, "achieved_gbs": gbs,
                     "frac": gbs / hbm})
    return rows


def issue_ceiling(entry, dom, clk_mhz: float, hbm: float):
    """Instruction-issue ceiling of the dominant kernel: its warp instructions per particle (ncu, on the kernel
    source recorded with them) at one warp instruction per cycle on each of the 4 schedulers of the 152 SMs."""
    if not entry or entry.get("kernel") != dom["kernel"] or not entry.get("warp_instructions_per_particle_step"):
        return None
    ipp = float(entry["warp_instructions_per_particle_step"])
    rate = 152 * 4 * clk_mhz * 1e6
    floor_ms = ipp * dom["particles"] / rate * 1e3
    return {"warp_instructions_per_particle": ipp, "issue_rate_per_s": rate, "floor_ms": floor_ms,
            "frac": floor_ms / dom["ms"] if dom["ms"] > 0 else None,
            "hbm_frac_at_floor": BYTES_PER_PARTICLE["f32"] * dom["particles"] / (floor_ms * 1e-3) / 1e9 / hbm, "sm_mhz": clk_mhz}


def run_ours(args):
    import torch

    import paper_2407_19151_gb300 as mcc

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device(f"cuda:{local}")
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    mcc.build()
    ctx = mcc.context(local)

    wl = make_workload(args.cells, rank, "f32", args.layout)
    N, C, S = wl.n, wl.n_cells, wl.n_species
    pairs = wl.pairs_per_step()
    species = list(zip(wl.q.tolist(), wl.m.tolist()))
    max_cell = int(wl.counts.sum(axis=1).max())
    params = mcc.Params(method=wl.method, dt=wl.dt, fE=wl.fE, seed=wl.seed, step=0)
    sharded = None
    if world > 1:
        # one global problem of world x C cells (rank r's block generated with its own seed), split by the
        # product's ShardedStep: rank r owns cells [r C, (r + 1) C), steps them with cell_base = r C, and the
        # per-species diagnostics are all-reduced after the timed steps
        from paper_2407_19151_gb300 import workloads as W
        from paper_2407_19151_gb300.sharding import ShardedStep
        counts = np.concatenate([W.three_species_counts(args.cells, data_seed=1239 + 1000 * r) for r in range(world)])
        goff = np.zeros(counts.size + 1, dtype=np.int64)
        np.cumsum(counts.ravel(), out=goff[1:])
        sharded = ShardedStep(goff, C * world, S, species, wl.lnL, params, max_cell=max_cell,
                              cell_range=(rank * C, (rank + 1) * C)).load(wl.vx, wl.vy, wl.vz, wl.w, local=True)
        params = sharded.params
        v, w, off = sharded.state["v"], sharded.state["w"], sharded.state["offsets"]
    else:
        off = torch.from_numpy(wl.offsets).to(dev)
        w = torch.from_numpy(wl.w).to(dev)
        v = [torch.from_numpy(np.ascontiguousarray(x)).to(dev) for x in (wl.vx, wl.vy, wl.vz)]
    corr = torch.zeros(C, dtype=torch.int32, device=dev)
    fail = torch.zeros(C, dtype=torch.int32, device=dev)

    def step(k0, nsteps=1):
        params.step = k0
        mcc.mcc_step_fused(*v, w, off, C, S, species, wl.lnL, params, n_steps=nsteps, max_cell=max_cell,
                           corr_pairs=corr, fail_count=fail)

    stream = torch.cuda.current_stream(dev)
    tuned = None
    if args.group_cap is None or args.tile_cap is None:
        tuned = mcc.autotune(*v, w, off, C, S, species, wl.lnL, params, max_cell)
    if args.group_cap is not None:
        ctx.set_group_capacity(args.group_cap)
    if args.tile_cap is not None:
        ctx.set_tile_cap(args.tile_cap)
    for k in range(args.warmup):
        step(k)
    torch.cuda.synchronize(dev)
    mcc.sync_status(local)

    # K steps captured in one CUDA graph, one mcc_step_fused call per step (cell order, queue reset, one kernel per
    # size class); each call records begin / end events around every class kernel as graph nodes, so that each
    # kernel's launches are timed on the stream they run on, inside the timed region
    n_ev = 2 * (mcc.GROUP_CLASSES + 1)
    events = [[torch.cuda.Event(enable_timing=True) for _ in range(n_ev)] for _ in range(args.steps)]
    for ev in events:
        for e in ev:
            e.record(stream)
    torch.cuda.synchronize(dev)
    g = torch.cuda.CUDAGraph()
    launches_before = ctx.launch_count()
    with torch.cuda.graph(g):
        for k in range(args.steps):
            params.launch_events = events[k]
            step(args.warmup + k)
    params.launch_events = None
    graph_launches = ctx.launch_count() - launches_before  # this library's kernels in the captured region
    torch.cuda.synchronize(dev)
    if world > 1:
        torch.distributed.barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        e0.record(stream)
        g.replay()
        e1.record(stream)
        torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1)
    class_ms = np.array([[ev[2 * c].elapsed_time(ev[2 * c + 1]) for c in range(mcc.GROUP_CLASSES + 1)]
                         for ev in events]).mean(axis=0)
    diagnostics = None
    if world > 1:
        t = torch.tensor([ms], device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        ms = float(t.item())
        diag, _ = sharded.diagnostics()  # the all-reduce of the per-species sums over the ranks
        diagnostics = {"particles": int(diag[:, 5].sum()), "weight": [float(x) for x in diag[:, 0]],
                       "kinetic_energy": [float(x) for x in diag[:, 4]]}
        torch.distributed.barrier()
    mcc.sync_status(local)
    ms_step = ms / args.steps
    value = pairs * world / (ms_step * 1e-3)
    hbm, peak_kind = peaks()
    fails = int(fail.sum().item())
    classes = class_table(wl, ctx.group_capacities(mcc.F32_MIXED, False), class_ms, hbm)
    dom = max(classes, key=lambda r: r["ms"])
    achieved = BYTES_PER_PARTICLE["f32"] * dom["particles"] / (dom["ms"] * 1e-3) / 1e9
    entry = ncu_entry("three_species")
    traffic = None
    if entry and entry.get("kernel") == dom["kernel"] and entry.get("bytes_per_particle"):
        traffic = entry["bytes_per_particle"] * dom["particles"]
    clocks = clk.summary()
    issue = issue_ceiling(entry, dom, clocks.get("sm_mhz") or 2070.0, hbm)

    # end to end through host buffers: every step copies its inputs in from pinned host memory and the updated
    # velocities back out, in cell chunks overlapped with the compute (host_pipeline.step_host, one round trip per
    # step, the pipeline kept full across steps); host wall clock around the call, synchronised
    e2e = None
    if not args.no_e2e:
        from paper_2407_19151_gb300.host_pipeline import step_host
        host = [torch.from_numpy(np.ascontiguousarray(x)).pin_memory() for x in (wl.vx, wl.vy, wl.vz)]
        host_w = torch.from_numpy(wl.w).pin_memory()
        e2e_steps = max(3, min(args.steps, 10))
        hp = mcc.Params(method=wl.method, dt=wl.dt, fE=wl.fE, seed=wl.seed, step=1000, cell_base=params.cell_base)
        step_host(*host, host_w, wl.offsets, C, S, species, wl.lnL, hp, n_steps=1, max_cell=max_cell,
                  chunks=args.e2e_chunks, buffers=args.e2e_buffers, device=local)
        torch.cuda.synchronize(dev)
        hp.step = 1001
        t0 = time.perf_counter()
        step_host(*host, host_w, wl.offsets, C, S, species, wl.lnL, hp, n_steps=1, max_cell=max_cell,
                  chunks=args.e2e_chunks, buffers=args.e2e_buffers, device=local, round_trips=e2e_steps)
        e_ms = (time.perf_counter() - t0) * 1e3 / e2e_steps
        bi = sum(h.numel() * h.element_size() for h in host) + host_w.numel() * 8
        bo = sum(h.numel() * h.element_size() for h in host)
        e2e = {"value": pairs * world / (e_ms * 1e-3), "unit": UNIT, "h2d_bytes_per_step": bi,
               "d2h_bytes_per_step": bo, "ms_per_step": e_ms, "chunks": args.e2e_chunks,
               "buffers": args.e2e_buffers, "steps": e2e_steps,
               "timing": "host wall clock around step_host: per step every chunk copied in, stepped and copied out; "
                         "synchronised at the end"}

    # plain FP64 GPU step on the same workload (the comparison point of the mixed path)
    fp64 = None
    if args.fp64_steps > 0:
        ctx.set_tile_cap(0)  # automatic tile for the double tile layout
        v64 = [torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64)).to(dev) for x in (wl.vx, wl.vy, wl.vz)]
        p64 = mcc.Params(method=wl.method, dt=wl.dt, fE=wl.fE, seed=wl.seed, step=0)
        mcc.mcc_step_fused(*v64, w, off, C, S, species, wl.lnL, p64, n_steps=1, max_cell=max_cell,
                           corr_pairs=corr, fail_count=fail)
        torch.cuda.synchronize(dev)
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        p64.step = 1
        mcc.mcc_step_fused(*v64, w, off, C, S, species, wl.lnL, p64, n_steps=args.fp64_steps, max_cell=max_cell,
                           corr_pairs=corr, fail_count=fail)
        f1.record(stream)
        torch.cuda.synchronize(dev)
        f_ms = f0.elapsed_time(f1) / args.fp64_steps
        fp64 = {"value": pairs * world / (f_ms * 1e-3), "unit": UNIT, "ms_per_step": f_ms,
                "roofline_frac_hbm": BYTES_PER_PARTICLE["f64"] * N / (f_ms * 1e-3) / 1e9 / hbm,
                "speedup_of_mixed": f_ms / ms_step}
        del v64
        mcc.sync_status(local)

    if rank != 0:
        return
    adj = None if (args.no_adjoint or world > 1) else adjoint_measure(dev)
    binning = None if (args.no_bin or world > 1) else bin_measure(wl, dev)
    other = None if (args.no_configs or world > 1) else configs_measure(dev, hbm)
    pic = None if (args.no_pic or world > 1) else pic_measure(wl, dev, hbm)
    cb = None if (args.no_cpu or world > 1) else cpu_baseline(wl, one_thread=True)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": bench_config(wl, args.layout, world),
        "launch": {"graph_steps": args.steps, "group_capacities": ctx.group_capacities(mcc.F32_MIXED, False),
                   "group_cap": args.group_cap if args.group_cap is not None else tuned["group_cap"],
                   "tile_cap": args.tile_cap if args.tile_cap is not None else tuned["tile_cap"],
                   "autotune": tuned, "precision": PRECISION},
        "roofline": {"bound": "hbm", "kernel": dom["kernel"], "achieved": achieved, "peak": hbm, "unit": "GB/s",
                     "frac": achieved / hbm, "traffic": traffic, "peak_kind": peak_kind,
                     "launch_ms": dom["ms"],
                     "algorithmic_bytes": f"{BYTES_PER_PARTICLE['f32']} B/particle x {dom['particles']} particles "
                                          f"per launch (the cells of its size class)",
                     "step": {"ms": ms_step, "achieved": BYTES_PER_PARTICLE["f32"] * N / (ms_step * 1e-3) / 1e9,
                              "frac": BYTES_PER_PARTICLE["f32"] * N / (ms_step * 1e-3) / 1e9 / hbm},
                     "classes": classes, "issue": issue,
                     "note": "instruction-issue- and latency-bound (per-cell barriers, dependent float-float "
                             "arithmetic), not HBM-bound"},
        "clocks": clocks,
        "e2e": e2e,
        "gpu_launches": graph_launches,  # one persistent step kernel per captured step + the cell-order kernel
        "correction_failures": fails,
        "sharded_diagnostics": diagnostics,
        "fp64_step": fp64,
        "adjoint": adj,
        "binning": binning,
        "other_workloads": other,
        "pic_coupling": pic,
        "cpu_baseline": cb,
    }
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
