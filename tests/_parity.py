"""Shared helpers of the GPU parity tests: move a seeded workload to the device, run the oracle on the same
inputs, and compare velocities relative to each (cell, species) population's rms speed."""
from __future__ import annotations

import numpy as np

import oracle as O
from paper_2407_19151_gb300 import workloads as W

F64_TOL = 1e-12   # FP64 path: relative velocity difference (spec tolerance)
F32_TOL = 2e-6    # mixed path: relative velocity difference (spec tolerance)


def device_state(wl: W.Workload, dtype: str, device="cuda:0"):
    import torch
    tdt = torch.float64 if dtype == "f64" else torch.float32
    v = [torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64)).to(device=device, dtype=tdt)
         for x in (wl.vx, wl.vy, wl.vz)]
    w = torch.from_numpy(np.ascontiguousarray(wl.w, dtype=np.float64)).to(device)
    off = torch.from_numpy(wl.offsets).to(device)
    return v, w, off


def oracle_state(wl: W.Workload, dtype: str) -> O.State:
    """FP64 oracle state from the same stored inputs (float32-rounded when the GPU stores floats)."""
    cast = (lambda x: np.asarray(x, dtype=np.float32).astype(np.float64)) if dtype == "f32" else \
        (lambda x: np.asarray(x, dtype=np.float64))
    return O.State(cast(wl.vx), cast(wl.vy), cast(wl.vz), wl.w, wl.offsets, wl.n_cells, wl.n_species)


def gpu_velocities(v) -> np.ndarray:
    return np.stack([x.double().cpu().numpy() for x in v], axis=1)


def population_scale(ref: np.ndarray, offsets: np.ndarray) -> np.ndarray:
    """Per particle: the rms speed of its (cell, species) population in the reference (floor: tiny)."""
    seg = np.diff(offsets)
    sp2 = (ref ** 2).sum(1)
    seg_id = np.repeat(np.arange(len(seg)), seg)
    sums = np.bincount(seg_id, weights=sp2, minlength=len(seg))
    rms = np.sqrt(sums / np.maximum(seg, 1))
    return np.maximum(rms[seg_id], 1e-300)


def velocity_error(got: np.ndarray, ref: np.ndarray, offsets: np.ndarray) -> np.ndarray:
    """Per-particle max-norm difference over the population rms speed."""
    return np.abs(got - ref).max(axis=1) / population_scale(ref, offsets)


def cell_moments(v: np.ndarray, w: np.ndarray, m, species: np.ndarray, offsets: np.ndarray, n_cells: int, S: int,
                 rel: bool = False, c: float = 1.0):
    """Per cell: momentum (3), kinetic energy, and the scales sum m w |v| and sum KE."""
    cells = np.repeat(np.arange(n_cells), np.diff(offsets[::S]))
    mp = np.asarray(m)[species] * w
    P = np.zeros((n_cells, 3))
    for d in range(3):
        np.add.at(P[:, d], cells, mp * v[:, d])
    v2 = (v ** 2).sum(1)
    ke = mp * v2 / (np.sqrt(1 + v2 / c ** 2) + 1) if rel else 0.5 * mp * v2
    E = np.zeros(n_cells)
    np.add.at(E, cells, ke)
    A = np.zeros(n_cells)
    np.add.at(A, cells, mp * np.sqrt(v2))
    return P, E, A
