"""Seeded synthetic plasmas for the collision step (inputs only; none of the method's arithmetic lives here).

Both the CUDA path and the oracle are fed from these generators. Units are normalised: electron mass,
elementary charge, vacuum permittivity and cell volume are 1 (so ``eps0 = dV = 1``) and ``c = 1`` where
relativistic. The time step is set from a reference collision frequency
``nu = q^4 lnL n / (4 pi eps0^2 m^2 v_t^3)`` of the electrons (``n`` the mean weighted density per cell,
``v_t = sqrt(T/m)`` with ``T`` the mean of the three axis temperatures) so that ``nu * dt`` is a small number.

The five workloads follow the paper's test plasmas (two-population relaxation, electron-ion thermalisation with
weighted particles; Secs. 5.1-5.3) scaled to GPU sizes:

1. ``isotropisation``  one electron species, 64 cells x 128, anisotropic Maxwellian Tx = 2 Ty = 2 Tz,
   weights log-uniform in [1, 10], lnL = 10, N97, FP64, nu*dt = 0.01.
2. ``equilibration``  electrons + ions (mass 100, Z = 1), 4096 cells, Poisson(256) particles per species per cell,
   electron weight 1, ion weights log-uniform in [10, 1000], T_e : T_i = 1 : 4, FP32 kinematics.
3. ``relativistic_beam``  beam electrons (u_z/c uniform so that gamma is in [2, 10], transverse spread 0.01c),
   thermal electrons and protons (T = 0.01 m_e c^2), 65536 cells with per-cell counts from a discrete power law
   N^-1.5 on [16, 2048] split 10 / 45 / 45, weights log-uniform over three decades.
4. ``differentiable``  electrons + protons (mass 1836), 1024 cells x 256 per species, T_e : T_p = 1 : 2,
   weights log-uniform in [1, 10].
5. ``three_species``  electrons, protons and C6+ ions (12 u - 6 m_e = 21868.66 m_e), 2^18 cells with log-normal
   per-cell counts (sigma 0.5, mean 512, about 1.34e8 particles), split evenly, weights log-uniform over four
   decades, T_e = 2 T_ion, N97, FP32 velocities with FP64 weights.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

TA77, N97 = 0, 1
AMU_IN_ME = 1822.888486
M_PROTON = 1836.15267
M_C6 = 12.0 * AMU_IN_ME - 6.0


@dataclass
class Workload:
    name: str
    n_cells: int
    q: np.ndarray
    m: np.ndarray
    lnL: np.ndarray
    counts: np.ndarray          # (n_cells, S) particles per cell and species
    vx: np.ndarray              # binned order (cell-major, then species)
    vy: np.ndarray
    vz: np.ndarray
    w: np.ndarray
    dt: float
    method: int = N97
    relativistic: bool = False
    fE: float = 0.05
    precision: str = "f64"      # "f64" or "f32" (velocity storage / kinematics)
    n_steps: int = 1
    seed: int = 0
    dV: float = 1.0
    eps0: float = 1.0
    c: float = 1.0
    meta: dict = field(default_factory=dict)

    @property
    def n_species(self) -> int:
        return len(self.m)

    @property
    def n(self) -> int:
        return int(self.counts.sum())

    @property
    def offsets(self) -> np.ndarray:
        off = np.zeros(self.n_cells * self.n_species + 1, dtype=np.int64)
        np.cumsum(self.counts.reshape(-1), out=off[1:])
        return off

    def species_of_particles(self) -> np.ndarray:
        return np.repeat(np.tile(np.arange(self.n_species, dtype=np.int32), self.n_cells),
                         self.counts.reshape(-1)).astype(np.int32)

    def cell_of_particles(self) -> np.ndarray:
        return np.repeat(np.arange(self.n_cells, dtype=np.int32), self.counts.sum(axis=1)).astype(np.int32)

    def interactions(self) -> np.ndarray:
        S = self.n_species
        return np.array([(a, b) for a in range(S) for b in range(a, S)], dtype=np.int32)

    def pairs_per_step(self) -> int:
        """Scatter-phase binary pairs of one step (a triplet counts as three), summed over interactions."""
        tot = 0
        cnt = self.counts.astype(np.int64)
        for a, b in self.interactions():
            if a == b:
                n = cnt[:, a]
                tot += int(np.where(n < 2, 0, np.where(n % 2 == 0, n // 2, (n + 3) // 2)).sum())
            else:
                na, nb = cnt[:, a], cnt[:, b]
                tot += int(np.where((na > 0) & (nb > 0), np.maximum(na, nb), 0).sum())
        return tot

    def weight_ordered(self) -> "Workload":
        """The same particles with each (cell, species) segment stored by descending weight (equal weights keep
        their order): the layout in which the optional weight order of the energy correction is the identity."""
        off = self.offsets
        seg = np.repeat(np.arange(len(off) - 1, dtype=np.int64), np.diff(off))
        # by segment, then descending weight, then index: a stable sort by weight, then a stable sort by segment.
        # Positive doubles order like their IEEE bit patterns read as int64, so both sorts are integer sorts (torch's
        # stable integer sort on the host is a radix sort, ~10x faster than numpy's at 1e8 particles).
        import torch
        by_w = torch.sort(torch.from_numpy(-np.ascontiguousarray(self.w).view(np.int64)), stable=True).indices
        seg_t = torch.from_numpy(seg)[by_w]
        order = by_w[torch.sort(seg_t, stable=True).indices].numpy()
        return Workload(self.name, self.n_cells, self.q, self.m, self.lnL, self.counts.copy(), self.vx[order],
                        self.vy[order], self.vz[order], self.w[order], self.dt, self.method, self.relativistic,
                        self.fE, self.precision, self.n_steps, self.seed, self.dV, self.eps0, self.c,
                        dict(self.meta, weight_ordered=True))

    def subset(self, n_cells: int) -> "Workload":
        """The first ``n_cells`` cells (cell ids, and hence every random draw, are unchanged)."""
        k = min(int(n_cells), self.n_cells)
        end = int(self.offsets[k * self.n_species])
        return Workload(self.name, k, self.q, self.m, self.lnL, self.counts[:k].copy(), self.vx[:end].copy(),
                        self.vy[:end].copy(), self.vz[:end].copy(), self.w[:end].copy(), self.dt, self.method,
                        self.relativistic, self.fE, self.precision, self.n_steps, self.seed, self.dV, self.eps0,
                        self.c, dict(self.meta))


def _loguniform(rng, lo_dec: float, hi_dec: float, n: int) -> np.ndarray:
    return 10.0 ** rng.uniform(lo_dec, hi_dec, n)


def _maxwellian(rng, n: int, T, m: float, drift=(0.0, 0.0, 0.0), dtype=np.float64):
    T = np.broadcast_to(np.asarray(T, dtype=np.float64), (3,))
    out = []
    for d in range(3):
        x = rng.standard_normal(n, dtype=np.float64) * np.sqrt(T[d] / m) + drift[d]
        out.append(x.astype(dtype))
    return out


def _dt_from_nu(nu_dt: float, q: float, m: float, lnL: float, n_mean: float, T_mean: float) -> float:
    v_t = np.sqrt(T_mean / m)
    nu = q ** 4 * lnL * n_mean / (4.0 * np.pi * m ** 2 * v_t ** 3)
    return nu_dt / nu


def _fill(rng, counts, species_spec, dtype):
    """Per (cell, species) segment, draw velocities and weights; species_spec[s] = (T, m, drift, wlo, whi) or a
    callable(rng, n) -> (vx, vy, vz, w)."""
    n_cells, S = counts.shape
    N = int(counts.sum())
    vx = np.empty(N, dtype=dtype); vy = np.empty(N, dtype=dtype); vz = np.empty(N, dtype=dtype)
    w = np.empty(N, dtype=np.float64)
    # draw per species over all cells at once, then scatter into binned (cell-major) order
    spec_of = np.tile(np.arange(S), n_cells)
    seg_len = counts.reshape(-1)
    seg_start = np.zeros_like(seg_len)
    np.cumsum(seg_len[:-1], out=seg_start[1:])
    for s in range(S):
        segs = np.nonzero(spec_of == s)[0]
        ns = int(seg_len[segs].sum())
        if ns == 0:
            continue
        spec = species_spec[s]
        if callable(spec):
            x, y, z, ww = spec(rng, ns)
        else:
            T, m, drift, wlo, whi = spec
            x, y, z = _maxwellian(rng, ns, T, m, drift, dtype)
            ww = _loguniform(rng, wlo, whi, ns) if whi > wlo else np.full(ns, 10.0 ** wlo)
        # destination indices of species s, in cell order
        idx = np.repeat(seg_start[segs] - np.concatenate([[0], np.cumsum(seg_len[segs])[:-1]]), seg_len[segs])
        idx = idx + np.arange(ns)
        vx[idx] = x; vy[idx] = y; vz[idx] = z; w[idx] = ww
    return vx, vy, vz, w


def isotropisation(n_cells: int = 64, per_cell: int = 128, data_seed: int = 1235, steps: int = 200) -> Workload:
    rng = np.random.default_rng(data_seed)
    counts = np.full((n_cells, 1), per_cell, dtype=np.int64)
    T = (2.0, 1.0, 1.0)
    vx, vy, vz, w = _fill(rng, counts, [(T, 1.0, (0, 0, 0), 0.0, 1.0)], np.float64)
    lnL = 10.0
    n_mean = float(np.mean(w)) * per_cell
    dt = _dt_from_nu(0.01, 1.0, 1.0, lnL, n_mean, np.mean(T))
    return Workload("isotropisation", n_cells, np.array([-1.0]), np.array([1.0]), np.full((1, 1), lnL), counts,
                    vx, vy, vz, w, dt, method=N97, precision="f64", n_steps=steps, seed=0x5EED0001,
                    meta={"T": T})


def equilibration(n_cells: int = 4096, mean_count: float = 256.0, data_seed: int = 1236, method: int = TA77,
                  precision: str = "f32", steps: int = 200) -> Workload:
    rng = np.random.default_rng(data_seed)
    counts = rng.poisson(mean_count, size=(n_cells, 2)).astype(np.int64)
    Te, Ti = 1.0, 4.0
    mi = 100.0
    vx, vy, vz, w = _fill(rng, counts, [(Te, 1.0, (0, 0, 0), 0.0, 0.0), (Ti, mi, (0, 0, 0), 1.0, 3.0)],
                          np.float64)
    lnL = 10.0
    dt = _dt_from_nu(0.01, 1.0, 1.0, lnL, mean_count * 1.0, Te)
    return Workload("equilibration", n_cells, np.array([-1.0, 1.0]), np.array([1.0, mi]), np.full((2, 2), lnL),
                    counts, vx, vy, vz, w, dt, method=method, precision=precision, n_steps=steps, seed=0x5EED0002,
                    meta={"T": (Te, Ti)})


def _power_law_counts(rng, n: int, lo: int, hi: int, alpha: float) -> np.ndarray:
    k = np.arange(lo, hi + 1, dtype=np.float64)
    p = k ** (-alpha)
    p /= p.sum()
    return rng.choice(np.arange(lo, hi + 1), size=n, p=p).astype(np.int64)


def relativistic_beam(n_cells: int = 65536, data_seed: int = 1237, steps: int = 100, count_lo: int = 16,
                      count_hi: int = 2048, precision: str = "f32") -> Workload:
    rng = np.random.default_rng(data_seed)
    tot = _power_law_counts(rng, n_cells, count_lo, count_hi, 1.5)
    nb = np.floor(0.10 * tot).astype(np.int64)
    ne = np.floor(0.45 * tot).astype(np.int64)
    npr = tot - nb - ne
    counts = np.stack([nb, ne, npr], axis=1)
    c = 1.0
    Tbg = 0.01

    def beam(rng_, n):
        uz = rng_.uniform(np.sqrt(3.0), np.sqrt(99.0), n) * c
        ux = rng_.standard_normal(n) * 0.01 * c
        uy = rng_.standard_normal(n) * 0.01 * c
        return ux, uy, uz, _loguniform(rng_, 0.0, 3.0, n)

    vx, vy, vz, w = _fill(rng, counts, [beam, (Tbg, 1.0, (0, 0, 0), 0.0, 3.0),
                                        (Tbg, M_PROTON, (0, 0, 0), 0.0, 3.0)], np.float64)
    lnL = 10.0
    w_mean = (10.0 ** 3 - 1.0) / (3.0 * np.log(10.0))
    dt = _dt_from_nu(0.01, 1.0, 1.0, lnL, float(np.mean(ne)) * w_mean, Tbg)
    return Workload("relativistic_beam", n_cells, np.array([-1.0, -1.0, 1.0]), np.array([1.0, 1.0, M_PROTON]),
                    np.full((3, 3), lnL), counts, vx, vy, vz, w, dt, method=N97, relativistic=True,
                    precision=precision, n_steps=steps, seed=0x5EED0003, c=c, meta={"T_bg": Tbg})


def differentiable(n_cells: int = 1024, per_species: int = 256, data_seed: int = 1238, steps: int = 50,
                   precision: str = "f64") -> Workload:
    rng = np.random.default_rng(data_seed)
    counts = np.full((n_cells, 2), per_species, dtype=np.int64)
    Te, Tp = 1.0, 2.0
    mp = 1836.0
    vx, vy, vz, w = _fill(rng, counts, [(Te, 1.0, (0, 0, 0), 0.0, 1.0), (Tp, mp, (0, 0, 0), 0.0, 1.0)],
                          np.float64)
    lnL = 10.0
    dt = _dt_from_nu(0.01, 1.0, 1.0, lnL, per_species * (9.0 / np.log(10.0)), Te)
    return Workload("differentiable", n_cells, np.array([-1.0, 1.0]), np.array([1.0, mp]), np.full((2, 2), lnL),
                    counts, vx, vy, vz, w, dt, method=N97, precision=precision, n_steps=steps, seed=0x5EED0004)


def _three_species_counts(rng, n_cells: int, mean_count: float, sigma: float) -> np.ndarray:
    mu = np.log(mean_count) - 0.5 * sigma * sigma
    tot = np.maximum(1, np.rint(np.exp(rng.normal(mu, sigma, n_cells)))).astype(np.int64)
    base = tot // 3
    rem = tot % 3
    return np.stack([base + (rem > 0), base + (rem > 1), base], axis=1).astype(np.int64)


def three_species_counts(n_cells: int = 1 << 18, mean_count: float = 512.0, sigma: float = 0.5,
                         data_seed: int = 1239) -> np.ndarray:
    """The (n_cells, 3) particle counts of three_species with the same arguments, without drawing the particles."""
    return _three_species_counts(np.random.default_rng(data_seed), n_cells, mean_count, sigma)


def three_species(n_cells: int = 1 << 18, mean_count: float = 512.0, sigma: float = 0.5, data_seed: int = 1239,
                  steps: int = 100, precision: str = "f32", method: int = N97) -> Workload:
    rng = np.random.default_rng(data_seed)
    counts = _three_species_counts(rng, n_cells, mean_count, sigma)
    Te, Ti = 1.0, 0.5
    dtype = np.float32 if precision == "f32" else np.float64
    vx, vy, vz, w = _fill(rng, counts, [(Te, 1.0, (0, 0, 0), 0.0, 4.0), (Ti, M_PROTON, (0, 0, 0), 0.0, 4.0),
                                        (Ti, M_C6, (0, 0, 0), 0.0, 4.0)], dtype)
    lnL = 10.0
    w_mean = (10.0 ** 4 - 1.0) / (4.0 * np.log(10.0))
    dt = _dt_from_nu(0.01, 1.0, 1.0, lnL, mean_count / 3.0 * w_mean, Te)
    return Workload("three_species", n_cells, np.array([-1.0, 1.0, 6.0]), np.array([1.0, M_PROTON, M_C6]),
                    np.full((3, 3), lnL), counts, vx, vy, vz, w, dt, method=method, precision=precision,
                    n_steps=steps, seed=0x5EED0005)


def grid_dims(n_cells: int) -> tuple[int, int, int]:
    """A near-cubic nx x ny x nz factorisation of n_cells (64^3 for 2^18 cells)."""
    n = int(n_cells)
    nz = max(d for d in range(1, int(round(n ** (1.0 / 3.0))) + 1) if n % d == 0)
    m = n // nz
    ny = max(d for d in range(1, int(m ** 0.5) + 1) if m % d == 0)
    return m // ny, ny, nz


def pic_setup(wl: Workload, cfl: float = 0.25, data_seed: int = 4242):
    """Positions for PIC coupling: the cells of ``wl`` on a periodic grid of unit cubes (volume dV = 1, cell id
    ix + nx (iy + ny iz)), each particle uniform inside its own cell, in the workload's precision. The push time
    step is set by a drift Courant number: ``cfl`` cell widths per step for the thermal speed of the lightest species
    (for a relativistic workload, for c), so that a fraction of the particles changes cell every step. Returns
    (grid, x, y, z, dt_push) with grid = ((nx, ny, nz), (lx, ly, lz))."""
    rng = np.random.default_rng(data_seed)
    nx, ny, nz = grid_dims(wl.n_cells)
    cell = wl.cell_of_particles().astype(np.int64)
    idx = (cell % nx, (cell // nx) % ny, cell // (nx * ny))
    dtype = np.float32 if wl.precision == "f32" else np.float64
    pos = []
    for i in idx:
        p = (i + rng.random(wl.n)).astype(dtype)
        top = np.nextafter((i + 1).astype(dtype), dtype(0))
        pos.append(np.minimum(p, top))   # rounding must not carry a particle into the next cell
    if wl.relativistic:
        v_t = wl.c
    else:
        light = int(np.argmin(wl.m))
        sp = wl.species_of_particles()
        v_t = float(np.sqrt(np.mean(np.asarray(wl.vx, dtype=np.float64)[sp == light] ** 2)))
    grid = ((nx, ny, nz), (float(nx), float(ny), float(nz)))
    return grid, pos[0], pos[1], pos[2], cfl / v_t


CONFIGS = {
    1: isotropisation,
    2: equilibration,
    3: relativistic_beam,
    4: differentiable,
    5: three_species,
}


def shuffled_order(n: int, data_seed: int = 99) -> np.ndarray:
    """A seeded random order of n particles (to hand unbinned particles to the binning call)."""
    return np.random.default_rng(data_seed).permutation(n).astype(np.int64)
