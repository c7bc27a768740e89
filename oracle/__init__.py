"""FP64 CPU oracle of the weighted, moment-preserving Monte-Carlo Coulomb collision step (ctypes wrapper).

TEST INFRASTRUCTURE ONLY. This package is the plain, slow reference that the CUDA library is checked against.
Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` import it; the product path
never does. It shares no code with ``paper_2407_19151_gb300``. The arithmetic lives in ``mcc_oracle.c``
(plain C, IEEE double, ``-ffp-contract=off``); this module only marshals numpy arrays.

Parity pins: see the header of ``mcc_oracle.h`` and ``tests/test_oracle_*.py``.
"""
from __future__ import annotations

import ctypes as C
import os
import platform
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mcc_oracle.c")
_HDR = os.path.join(_HERE, "mcc_oracle.h")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, f"libmcc_oracle.{platform.machine()}.so")

TA77, N97 = 0, 1
FAIL_ROLLBACK, FAIL_MOMENTUM_ONLY, FAIL_ERROR = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/_build`` (gcc, C11, -O2 -ffp-contract=off -fopenmp)."""
    os.makedirs(_BUILD, exist_ok=True)
    newest_src = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= newest_src:
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Params(C.Structure):
    _fields_ = [
        ("method", C.c_int32), ("relativistic", C.c_int32),
        ("dt", C.c_double), ("dV", C.c_double), ("eps0", C.c_double), ("c", C.c_double), ("fE", C.c_double),
        ("sort_by_weight", C.c_int32), ("max_corr_passes", C.c_int32), ("fail_policy", C.c_int32),
        ("correct", C.c_int32), ("seed", C.c_uint64), ("step", C.c_uint64), ("weighting", C.c_int32),
        ("pairing", C.c_int32),
    ]


@dataclass
class Params:
    """Step parameters (mirrors ``orc_params``)."""
    method: int = N97
    relativistic: bool = False
    dt: float = 1.0
    dV: float = 1.0
    eps0: float = 1.0
    c: float = 1.0
    fE: float = 0.05
    sort_by_weight: bool = True
    max_corr_passes: int = 8
    fail_policy: int = FAIL_ROLLBACK
    correct: bool = True
    seed: int = 0
    step: int = 0
    weighting: int = 0   # 0: the paper's s; 1: duplicity weighting (w_max / D_ij, N_max) for inter-species pairs
    pairing: int = 0     # 0: order-N pairs (Eq. sab_TA77); 1: all N x N pairs (Eq. sab_weighted)

    def _c(self) -> _Params:
        return _Params(int(self.method), int(bool(self.relativistic)), float(self.dt), float(self.dV),
                       float(self.eps0), float(self.c), float(self.fE), int(bool(self.sort_by_weight)),
                       int(self.max_corr_passes), int(self.fail_policy), int(bool(self.correct)),
                       int(self.seed) & (2**64 - 1), int(self.step) & (2**64 - 1), int(self.weighting),
                       int(self.pairing))


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        P = C.POINTER
        d, i32, i64, u8, u32 = P(C.c_double), P(C.c_int32), P(C.c_int64), P(C.c_uint8), P(C.c_uint32)
        sig = {
            "orc_philox4x32_10": (None, [u32, u32, u32]),
            "orc_bin": (C.c_int, [i32, i32, C.c_int64, C.c_int32, C.c_int32, i32, i64]),
            "orc_set_threads": (None, [C.c_int32]),
            "orc_push": (C.c_int, [C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                   C.c_int64, i32, d, C.c_double, C.c_int32, C.c_double, i32]),
            "orc_nxn_slot": (C.c_int, [C.c_int64, C.c_int64, C.c_int32, C.c_int64, i64, i64]),
            "orc_nxn_slots": (C.c_int64, [C.c_int64, C.c_int64, C.c_int32, i64]),
            "orc_bin_weighted": (C.c_int, [i32, i32, d, C.c_int64, C.c_int32, C.c_int32, i32, i64]),
            "orc_permutation": (C.c_int, [C.c_int64, C.c_uint64, C.c_uint64, C.c_uint32, C.c_uint32, C.c_uint32,
                                          i32]),
            "orc_pairs": (C.c_int, [i64, C.c_int32, C.c_int32, C.c_int32, C.c_int32, C.c_int32, C.c_uint64,
                                    C.c_uint64, i32, i32, u8]),
            "orc_n97_A": (C.c_double, [C.c_double]),
            "orc_n97_L": (C.c_double, [C.c_double]),
            "orc_angle": (None, [C.c_int32, C.c_double, C.c_double, C.c_double, d, d]),
            "orc_rotate": (None, [d, C.c_double, C.c_double, C.c_double, d]),
            "orc_energy_pair": (None, [C.c_int32, C.c_double, C.c_double, C.c_double, d, d, C.c_double]),
            "orc_pair_kecm": (C.c_double, [C.c_int32, C.c_double, C.c_double, C.c_double, d, d]),
            "orc_rel_scatter_dp": (None, [C.c_double, C.c_double, C.c_double, d, d, C.c_double, C.c_double,
                                          C.c_double, d, d, d]),
            "orc_scatter": (C.c_int, [d, d, d, d, i64, C.c_int32, C.c_int32, d, d, d, C.c_int32, C.c_int32,
                                      C.c_int32, P(_Params), d]),
            "orc_correct": (C.c_int, [d, d, d, d, i64, C.c_int32, C.c_int32, d, C.c_int32, C.c_int32, C.c_int32,
                                      P(_Params), d, i32, i32]),
            "orc_step": (C.c_int, [d, d, d, d, i64, C.c_int32, C.c_int32, d, d, d, i32, C.c_int32, P(_Params),
                                   C.c_int32, C.c_int32, C.c_int32, i32, i32]),
        }
        for name, (res, args) in sig.items():
            f = getattr(_lib, name)
            f.restype = res
            f.argtypes = args
    return _lib


def _p(a, ctype):
    return a.ctypes.data_as(C.POINTER(ctype))


def _check(rc, what):
    if rc != 0:
        raise ValueError(f"oracle {what} failed with code {rc}")


# ---------------------------------------------------------------------------------------------- small pieces
def philox4x32_10(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().orc_philox4x32_10(_p(c, C.c_uint32), _p(k, C.c_uint32), _p(out, C.c_uint32))
    return out


def nxn_schedule(na: int, nb: int, intra: bool):
    """The order N x N schedule of one cell: list of (slot, round, local a, local b) before the permutations."""
    per = np.zeros(1, dtype=np.int64)
    n = lib().orc_nxn_slots(na, nb, int(intra), _p(per, C.c_int64))
    out = []
    a = np.zeros(1, dtype=np.int64)
    b = np.zeros(1, dtype=np.int64)
    for k in range(n):
        if lib().orc_nxn_slot(na, nb, int(intra), k, _p(a, C.c_int64), _p(b, C.c_int64)):
            out.append((k, k // int(per[0]), int(a[0]), int(b[0])))
    return out


def set_threads(n: int):
    """Host threads used by step() (timing only)."""
    lib().orc_set_threads(int(n))


def push(x, y, z, vx, vy, vz, grid, dt: float, relativistic: bool = False, c: float = 1.0):
    """Free-streaming push in a periodic box (see orc_push), in the precision of the given arrays (float64 or
    float32, all alike). ``grid`` = ((nx, ny, nz), (lx, ly, lz)). Returns (x, y, z, cell) as new arrays."""
    (nx, ny, nz), (lx, ly, lz) = grid
    dt_ = np.asarray(vx).dtype
    if dt_ not in (np.float64, np.float32):
        raise TypeError("float64 or float32 arrays")
    arrs = [np.array(a, dtype=dt_, copy=True) for a in (x, y, z)]
    vel = [np.ascontiguousarray(a, dtype=dt_) for a in (vx, vy, vz)]
    n = len(vel[0])
    cell = np.zeros(n, dtype=np.int32)
    nc = np.array([nx, ny, nz], dtype=np.int32)
    l = np.array([lx, ly, lz], dtype=np.float64)
    vp = [a.ctypes.data_as(C.c_void_p) for a in arrs + vel]
    _check(lib().orc_push(0 if dt_ == np.float64 else 1, *vp, n, _p(nc, C.c_int32), _p(l, C.c_double), float(dt),
                          int(bool(relativistic)), float(c), _p(cell, C.c_int32)), "push")
    return arrs[0], arrs[1], arrs[2], cell


def bin_particles(cell, species, n_cells: int, n_species: int):
    cell = np.ascontiguousarray(cell, dtype=np.int32)
    species = np.ascontiguousarray(species, dtype=np.int32)
    perm = np.zeros(len(cell), dtype=np.int32)
    offsets = np.zeros(n_cells * n_species + 1, dtype=np.int64)
    _check(lib().orc_bin(_p(cell, C.c_int32), _p(species, C.c_int32), len(cell), n_cells, n_species,
                         _p(perm, C.c_int32), _p(offsets, C.c_int64)), "bin")
    return perm, offsets


def bin_particles_weighted(cell, species, w, n_cells: int, n_species: int):
    """Cell sort with every segment in the weight-sort order of Algorithm 1 (see orc_bin_weighted)."""
    cell = np.ascontiguousarray(cell, dtype=np.int32)
    species = np.ascontiguousarray(species, dtype=np.int32)
    w = np.ascontiguousarray(w, dtype=np.float64)
    perm = np.zeros(len(cell), dtype=np.int32)
    offsets = np.zeros(n_cells * n_species + 1, dtype=np.int64)
    _check(lib().orc_bin_weighted(_p(cell, C.c_int32), _p(species, C.c_int32), _p(w, C.c_double), len(cell),
                                  n_cells, n_species, _p(perm, C.c_int32), _p(offsets, C.c_int64)), "bin_weighted")
    return perm, offsets


def permutation(n: int, seed: int, step: int, cell: int, inter: int, side: int) -> np.ndarray:
    out = np.zeros(max(n, 1), dtype=np.int32)
    _check(lib().orc_permutation(n, seed, step, cell, inter, side, _p(out, C.c_int32)), "permutation")
    return out[:n]


def pairs(offsets, n_cells: int, n_species: int, sa: int, sb: int, inter: int, seed: int, step: int):
    offsets = np.ascontiguousarray(offsets, dtype=np.int64)
    N = int(offsets[-1])
    pi = np.full(max(N, 1), -1, dtype=np.int32)
    pj = np.full(max(N, 1), -1, dtype=np.int32)
    fl = np.zeros(max(N, 1), dtype=np.uint8)
    _check(lib().orc_pairs(_p(offsets, C.c_int64), n_cells, n_species, sa, sb, inter, seed, step,
                           _p(pi, C.c_int32), _p(pj, C.c_int32), _p(fl, C.c_uint8)), "pairs")
    return pi[:N], pj[:N], fl[:N]


def n97_A(s: float) -> float:
    return lib().orc_n97_A(float(s))


def n97_L(A: float) -> float:
    return lib().orc_n97_L(float(A))


def angle(method: int, s: float, U1: float, U4: float):
    st, omc = C.c_double(), C.c_double()
    lib().orc_angle(method, s, U1, U4, C.byref(st), C.byref(omc))
    return st.value, omc.value


def rotate(u, sin_theta: float, one_minus_cos: float, phi: float) -> np.ndarray:
    u = np.ascontiguousarray(u, dtype=np.float64)
    du = np.zeros(3)
    lib().orc_rotate(_p(u, C.c_double), sin_theta, one_minus_cos, phi, _p(du, C.c_double))
    return du


def energy_pair(relativistic: bool, c: float, m1: float, m2: float, v1, v2, U: float):
    a = np.array(v1, dtype=np.float64)
    b = np.array(v2, dtype=np.float64)
    lib().orc_energy_pair(int(relativistic), c, m1, m2, _p(a, C.c_double), _p(b, C.c_double), U)
    return a, b


def pair_kecm(relativistic: bool, c: float, m1: float, m2: float, v1, v2) -> float:
    a = np.ascontiguousarray(v1, dtype=np.float64)
    b = np.ascontiguousarray(v2, dtype=np.float64)
    return lib().orc_pair_kecm(int(relativistic), c, m1, m2, _p(a, C.c_double), _p(b, C.c_double))


def rel_scatter_dp(c, ma, mb, ui, uj, sin_theta, one_minus_cos, phi):
    ui = np.ascontiguousarray(ui, dtype=np.float64)
    uj = np.ascontiguousarray(uj, dtype=np.float64)
    dp = np.zeros(3)
    pm, vr = C.c_double(), C.c_double()
    lib().orc_rel_scatter_dp(c, ma, mb, _p(ui, C.c_double), _p(uj, C.c_double), sin_theta, one_minus_cos, phi,
                             _p(dp, C.c_double), C.byref(pm), C.byref(vr))
    return dp, pm.value, vr.value


# ---------------------------------------------------------------------------------------------- whole arrays
class State:
    """Binned FP64 particle state: contiguous copies of vx, vy, vz, w plus segment offsets (cell-major)."""

    def __init__(self, vx, vy, vz, w, offsets, n_cells: int, n_species: int):
        self.vx = np.array(vx, dtype=np.float64)
        self.vy = np.array(vy, dtype=np.float64)
        self.vz = np.array(vz, dtype=np.float64)
        self.w = np.ascontiguousarray(w, dtype=np.float64)
        self.offsets = np.ascontiguousarray(offsets, dtype=np.int64)
        self.n_cells = int(n_cells)
        self.n_species = int(n_species)

    @property
    def n(self) -> int:
        return int(self.offsets[-1])

    def v(self) -> np.ndarray:
        return np.stack([self.vx, self.vy, self.vz], axis=1)


def _species_arrays(q, m, lnL, S):
    q = np.ascontiguousarray(q, dtype=np.float64)
    m = np.ascontiguousarray(m, dtype=np.float64)
    L = np.asarray(lnL, dtype=np.float64)
    if L.ndim == 0:
        L = np.full((S, S), float(L))
    L = np.ascontiguousarray(L.reshape(S, S))
    return q, m, L


def scatter(st: State, q, m, lnL, sa: int, sb: int, inter: int, p: Params) -> np.ndarray:
    """Scatter of interaction (sa, sb) in every cell; returns the pre-scatter copy (3, N)."""
    q, m, L = _species_arrays(q, m, lnL, st.n_species)
    backup = np.zeros((3, max(st.n, 1)))
    cp = p._c()
    _check(lib().orc_scatter(_p(st.vx, C.c_double), _p(st.vy, C.c_double), _p(st.vz, C.c_double),
                             _p(st.w, C.c_double), _p(st.offsets, C.c_int64), st.n_cells, st.n_species,
                             _p(q, C.c_double), _p(m, C.c_double), _p(L, C.c_double), sa, sb, inter, C.byref(cp),
                             _p(backup, C.c_double)), "scatter")
    return backup[:, : st.n] if st.n else backup[:, :0]


def correct(st: State, m, sa: int, sb: int, inter: int, p: Params, backup: np.ndarray):
    """Moment correction of interaction (sa, sb) in every cell; returns (corr_pairs, fail_flags) per cell."""
    m = np.ascontiguousarray(m, dtype=np.float64)
    bk = np.zeros((3, max(st.n, 1)))
    bk[:, : st.n] = backup
    corr = np.zeros(st.n_cells, dtype=np.int32)
    fail = np.zeros(st.n_cells, dtype=np.int32)
    cp = p._c()
    _check(lib().orc_correct(_p(st.vx, C.c_double), _p(st.vy, C.c_double), _p(st.vz, C.c_double),
                             _p(st.w, C.c_double), _p(st.offsets, C.c_int64), st.n_cells, st.n_species,
                             _p(m, C.c_double), sa, sb, inter, C.byref(cp), _p(bk, C.c_double),
                             _p(corr, C.c_int32), _p(fail, C.c_int32)), "correct")
    return corr, fail


def default_interactions(n_species: int) -> np.ndarray:
    """Interaction list in lexicographic order (a <= b): (0,0), (0,1), ..., (1,1), ..."""
    return np.array([(a, b) for a in range(n_species) for b in range(a, n_species)], dtype=np.int32)


def step(st: State, q, m, lnL, p: Params, n_steps: int = 1, interactions=None, cell_begin: int = 0,
         cell_end: int | None = None):
    """n_steps full collision steps on cells [cell_begin, cell_end); returns (corr_pairs, fail_count) per cell."""
    q, m, L = _species_arrays(q, m, lnL, st.n_species)
    inter = default_interactions(st.n_species) if interactions is None else np.ascontiguousarray(
        interactions, dtype=np.int32).reshape(-1, 2)
    corr = np.zeros(st.n_cells, dtype=np.int32)
    fail = np.zeros(st.n_cells, dtype=np.int32)
    cp = p._c()
    ce = st.n_cells if cell_end is None else int(cell_end)
    _check(lib().orc_step(_p(st.vx, C.c_double), _p(st.vy, C.c_double), _p(st.vz, C.c_double),
                          _p(st.w, C.c_double), _p(st.offsets, C.c_int64), st.n_cells, st.n_species,
                          _p(q, C.c_double), _p(m, C.c_double), _p(L, C.c_double),
                          _p(np.ascontiguousarray(inter), C.c_int32), len(inter), C.byref(cp), int(n_steps),
                          int(cell_begin), ce, _p(corr, C.c_int32), _p(fail, C.c_int32)), "step")
    return corr, fail
