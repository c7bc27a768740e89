"""Thin ctypes binding of the C ABI in ``include/mcc.h``: argument marshalling between torch CUDA tensors and the
library. Every step of the collision method runs in the CUDA library; nothing here computes on particles. If the
library is not built the calls raise (there is no CPU fallback)."""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import torch

from . import _build

TA77, N97 = 0, 1
F64, F32_MIXED = 0, 1
FAIL_ROLLBACK, FAIL_MOMENTUM_ONLY, FAIL_ERROR = 0, 1, 2

STATUS = {0: "ok", -1: "invalid argument", -2: "CUDA error", -3: "workspace missing or too small",
          -4: "bounded wait timed out", -5: "energy correction could not absorb the violation",
          -6: "index or cell size out of bounds", -7: "segment larger than supported"}


class MccError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"{what}: {STATUS.get(code, 'unknown')} ({code})")
        self.code = code


class _Species(C.Structure):
    _fields_ = [("q", C.c_double), ("m", C.c_double)]


class _Particles(C.Structure):
    _fields_ = [("vx", C.c_void_p), ("vy", C.c_void_p), ("vz", C.c_void_p), ("w", C.c_void_p),
                ("n", C.c_int64), ("prec", C.c_int32)]


class _Grid(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32), ("lx", C.c_double), ("ly", C.c_double),
                ("lz", C.c_double)]


class _Params(C.Structure):
    _fields_ = [("method", C.c_int32), ("relativistic", C.c_int32), ("dt", C.c_double), ("dV", C.c_double),
                ("eps0", C.c_double), ("c", C.c_double), ("fE", C.c_double), ("sort_by_weight", C.c_int32),
                ("max_corr_passes", C.c_int32), ("fail_policy", C.c_int32), ("correct", C.c_int32),
                ("seed", C.c_uint64), ("step", C.c_uint64), ("cell_base", C.c_uint32),
                ("weighting", C.c_int32), ("pairing", C.c_int32), ("step_device", C.c_void_p),
                ("residual", C.c_void_p), ("launch_events", C.c_void_p)]


@dataclass
class Params:
    """Mirror of ``mcc_params``."""
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
    cell_base: int = 0
    weighting: int = 0   # 0: the paper's s; 1: duplicity weighting (w_max / D_ij, N_max) for inter-species pairs
    pairing: int = 0     # 0: order-N pairs; 1: all N x N pairs (fused step only)
    step_device: object = None  # optional int64/uint64 device tensor of one element holding the step (fused step)
    residual: object = None     # optional float64 device tensor (2 * n_cells): per-cell conservation of the on-chip
                                # state before the store (fused step)
    launch_events: object = None  # optional list of 2 (GROUP_CLASSES + 1) torch.cuda.Event(enable_timing=True):
                                  # begin / end of each size class's kernel in the last step (fused step)

    def _c(self) -> _Params:
        return _Params(int(self.method), int(bool(self.relativistic)), float(self.dt), float(self.dV),
                       float(self.eps0), float(self.c), float(self.fE), int(bool(self.sort_by_weight)),
                       int(self.max_corr_passes), int(self.fail_policy), int(bool(self.correct)),
                       int(self.seed) & (2**64 - 1), int(self.step) & (2**64 - 1), int(self.cell_base),
                       int(self.weighting), int(self.pairing),
                       C.c_void_p(self.step_device.data_ptr()) if self.step_device is not None else C.c_void_p(0),
                       C.c_void_p(self.residual.data_ptr()) if self.residual is not None else C.c_void_p(0),
                       _events(self.launch_events))


GROUP_CLASSES = 5  # size classes of the group kernels (MCC_GROUP_CLASSES)
_LIB = None
_EVENT_ARRAYS = []


def _events(events):
    """Host array of the cudaEvent_t handles of a list of torch CUDA events (kept alive with the last call)."""
    if events is None:
        return C.c_void_p(0)
    for e in events:
        if e.cuda_event == 0:  # created lazily by torch: record once so that the handle exists
            e.record()
    arr = (C.c_void_p * len(events))(*[e.cuda_event for e in events])
    _EVENT_ARRAYS[:] = [arr]
    return C.cast(arr, C.c_void_p)


def lib():
    """The loaded CUDA library; raises if it has not been built (no fallback)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = os.environ.get("MCC_LIBRARY") or _build.lib_path()
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library not built ({path}); run paper_2407_19151_gb300.build()")
    L = C.CDLL(path)
    P, vp = C.POINTER, C.c_void_p
    sig = {
        "mcc_create": (C.c_int, [P(vp), C.c_int]),
        "mcc_destroy": (None, [vp]),
        "mcc_bin_workspace_size": (C.c_int, [C.c_int64, C.c_int32, C.c_int32, P(C.c_size_t)]),
        "mcc_bin": (C.c_int, [vp, vp, vp, C.c_int64, C.c_int32, C.c_int32, vp, vp, vp, C.c_size_t, vp]),
        "mcc_adjoint_workspace_size": (C.c_int, [vp, C.c_int32, C.c_int32, C.c_int32, P(C.c_size_t)]),
        "mcc_adjoint_tape_size": (C.c_int, [vp, C.c_int32, C.c_int32, C.c_int32, P(C.c_size_t)]),
        "mcc_adjoint": (C.c_int, [vp, P(_Particles), vp, C.c_int32, C.c_int32, P(_Species), P(C.c_double), C.c_int32,
                                  C.c_int32, C.c_int32, P(_Params), C.c_int32, vp, vp, vp, vp, vp, vp, vp, vp,
                                  C.c_int32, vp, C.c_size_t, vp]),
        "mcc_bin_weighted_workspace_size": (C.c_int, [C.c_int64, C.c_int32, C.c_int32, P(C.c_size_t)]),
        "mcc_bin_weighted": (C.c_int, [vp, vp, vp, vp, C.c_int64, C.c_int32, C.c_int32, vp, vp, vp, C.c_size_t,
                                       vp]),
        "mcc_gather": (C.c_int, [vp, vp, C.c_int64, C.c_int32, vp, vp]),
        "mcc_species_moments": (C.c_int, [vp, P(_Particles), vp, C.c_int32, C.c_int32, P(_Species), C.c_int32,
                                          C.c_double, vp, vp, vp]),
        "mcc_gather_n": (C.c_int, [P(vp), P(vp), P(C.c_int32), C.c_int32, vp, C.c_int64, vp]),
        "mcc_push": (C.c_int, [P(_Particles), vp, vp, vp, P(_Grid), C.c_double, C.c_int32, C.c_double, vp, vp]),
        "mcc_bin_static": (C.c_int, [vp, vp, C.c_int64, C.c_int32, C.c_int32, vp, vp, vp]),
        "mcc_pair": (C.c_int, [vp, vp, C.c_int32, C.c_int32, C.c_int32, C.c_int32, C.c_int32, C.c_uint64,
                               C.c_uint64, vp, vp, vp, vp]),
        "mcc_scatter": (C.c_int, [vp, P(_Particles), vp, C.c_int32, C.c_int32, P(_Species), P(C.c_double),
                                  C.c_int32, C.c_int32, C.c_int32, vp, vp, vp, P(_Params), vp, vp]),
        "mcc_correct": (C.c_int, [vp, P(_Particles), vp, C.c_int32, C.c_int32, P(_Species), C.c_int32,
                                  C.c_int32, C.c_int32, P(_Params), vp, vp, vp, vp]),
        "mcc_step_workspace_size": (C.c_int, [vp, C.c_int32, C.c_int32, C.c_int32, P(C.c_size_t)]),
        "mcc_step_fused": (C.c_int, [vp, P(_Particles), vp, C.c_int32, C.c_int32, P(_Species), P(C.c_double),
                                     P(C.c_int32), C.c_int32, P(_Params), C.c_int32, C.c_int32, vp, vp, vp,
                                     C.c_size_t, vp]),
        "mcc_set_tile_cap": (C.c_int, [vp, C.c_int32]),
        "mcc_set_group_capacity": (C.c_int, [vp, C.c_int32, C.c_int32]),
        "mcc_group_capacities": (C.c_int, [vp, C.c_int32, C.c_int32, P(C.c_int32)]),
        "mcc_sync_status": (C.c_int, [vp, vp]),
        "mcc_launch_count": (C.c_int64, [vp]),
        "mcc_debug_record": (C.c_int, [vp, vp, P(C.c_int32)]),
        "mcc_debug_bounds_build": (C.c_int, []),
        "mcc_phase_clocks": (C.c_int, [vp, vp, P(C.c_uint64)]),
        "mcc_phase_clocks_build": (C.c_int, []),
        "mcc_status_string": (C.c_char_p, [C.c_int]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _LIB = L
    return L


def _check(rc: int, what: str):
    if rc != 0:
        raise MccError(rc, what)


class Context:
    """An ``mcc_ctx`` on one device (status word, work-queue counter) plus cached workspaces."""

    def __init__(self, device: int = 0):
        self.device = int(device)
        h = C.c_void_p()
        _check(lib().mcc_create(C.byref(h), self.device), "mcc_create")
        self.handle = h
        self._ws = {}

    def __del__(self):
        try:
            if self.handle:
                lib().mcc_destroy(self.handle)
        except Exception:
            pass

    def workspace(self, key, nbytes: int) -> torch.Tensor | None:
        if nbytes == 0:
            return None
        t = self._ws.get(key)
        if t is None or t.numel() < nbytes:
            t = torch.empty(nbytes, dtype=torch.uint8, device=f"cuda:{self.device}")
            self._ws[key] = t
        return t

    def launch_count(self) -> int:
        return int(lib().mcc_launch_count(self.handle))

    def set_tile_cap(self, cap: int):
        _check(lib().mcc_set_tile_cap(self.handle, int(cap)), "mcc_set_tile_cap")

    def set_group_capacity(self, particles_per_warp: int, largest: int = 0):
        _check(lib().mcc_set_group_capacity(self.handle, int(particles_per_warp), int(largest)),
               "mcc_set_group_capacity")

    def group_capacities(self, prec: int = F32_MIXED, relativistic: bool = False) -> list[int]:
        caps = (C.c_int32 * GROUP_CLASSES)()
        _check(lib().mcc_group_capacities(self.handle, int(prec), int(bool(relativistic)), caps),
               "mcc_group_capacities")
        return list(caps)

    def debug_record(self, stream=None) -> list[int]:
        """(source line, index, bound, count) of the first out-of-bounds index seen by a bounds-checked build."""
        out = (C.c_int32 * 4)()
        _check(lib().mcc_debug_record(self.handle, _stream(stream, self.device), out), "mcc_debug_record")
        return list(out)

    def phase_clocks(self, stream=None) -> list[list[int]]:
        """Per group size class: cycles of the 7 phases of a cell visit and the number of visits (phase-timing
        builds; zeros otherwise)."""
        out = (C.c_uint64 * 40)()
        _check(lib().mcc_phase_clocks(self.handle, _stream(stream, self.device), out), "mcc_phase_clocks")
        return [list(out[8 * k: 8 * k + 8]) for k in range(5)]

    def sync_status(self, stream=None) -> int:
        return int(lib().mcc_sync_status(self.handle, _stream(stream, self.device)))


_CTX: dict[int, Context] = {}


def context(device: int | torch.device | None = None) -> Context:
    dev = torch.cuda.current_device() if device is None else torch.device(device).index or 0
    if dev not in _CTX:
        _CTX[dev] = Context(dev)
    return _CTX[dev]


def _stream(stream, device):
    if stream is None:
        stream = torch.cuda.current_stream(device)
    return C.c_void_p(stream.cuda_stream)


def _ptr(t: torch.Tensor | None):
    return C.c_void_p(t.data_ptr()) if t is not None else C.c_void_p(0)


def _particles(vx, vy, vz, w) -> _Particles:
    if vx.dtype == torch.float64:
        prec = F64
    elif vx.dtype == torch.float32:
        prec = F32_MIXED
    else:
        raise TypeError("velocities must be float64 or float32")
    for t in (vx, vy, vz):
        if t.dtype != vx.dtype or not t.is_cuda or not t.is_contiguous() or t.numel() != vx.numel():
            raise TypeError("vx, vy, vz must be contiguous CUDA tensors of one dtype and length")
    if w.dtype != torch.float64 or not w.is_cuda or not w.is_contiguous() or w.numel() != vx.numel():
        raise TypeError("w must be a contiguous float64 CUDA tensor of the particles' length")
    return _Particles(vx.data_ptr(), vy.data_ptr(), vz.data_ptr(), w.data_ptr(), vx.numel(), prec)


def _species(species) -> C.Array:
    arr = (_Species * len(species))()
    for k, (q, m) in enumerate(species):
        arr[k] = _Species(float(q), float(m))
    return arr


def _lnL(lnL, S: int):
    import numpy as np
    L = np.asarray(lnL, dtype=np.float64)
    if L.ndim == 0:
        L = np.full((S, S), float(L))
    L = np.ascontiguousarray(L.reshape(S, S))
    return (C.c_double * (S * S))(*L.reshape(-1).tolist())


# ---------------------------------------------------------------------------------------------------- C-ABI calls
def mcc_bin(cell: torch.Tensor, species: torch.Tensor, n_cells: int, n_species: int, stream=None):
    """Stable counting sort by (cell, species); returns (perm int32[n], offsets int64[n_cells*n_species+1])."""
    ctx = context(cell.device)
    n = cell.numel()
    perm = torch.empty(n, dtype=torch.int32, device=cell.device)
    offsets = torch.empty(n_cells * n_species + 1, dtype=torch.int64, device=cell.device)
    nb = C.c_size_t()
    _check(lib().mcc_bin_workspace_size(n, n_cells, n_species, C.byref(nb)), "mcc_bin_workspace_size")
    ws = ctx.workspace("bin", nb.value)
    _check(lib().mcc_bin(ctx.handle, _ptr(cell), _ptr(species), n, n_cells, n_species, _ptr(perm), _ptr(offsets),
                         _ptr(ws), nb.value, _stream(stream, cell.device)), "mcc_bin")
    return perm, offsets


def mcc_bin_weighted(cell: torch.Tensor, species: torch.Tensor, w: torch.Tensor, n_cells: int, n_species: int,
                     stream=None):
    """Cell sort with each segment in descending-weight order (ties by index); outputs as mcc_bin."""
    ctx = context(cell.device)
    n = cell.numel()
    if w.dtype != torch.float64 or w.numel() != n:
        raise ValueError("w must be float64 with one weight per particle")
    perm = torch.empty(n, dtype=torch.int32, device=cell.device)
    offsets = torch.empty(n_cells * n_species + 1, dtype=torch.int64, device=cell.device)
    nb = C.c_size_t()
    _check(lib().mcc_bin_weighted_workspace_size(n, n_cells, n_species, C.byref(nb)),
           "mcc_bin_weighted_workspace_size")
    ws = ctx.workspace("bin_weighted", nb.value)
    _check(lib().mcc_bin_weighted(ctx.handle, _ptr(cell), _ptr(species), _ptr(w), n, n_cells, n_species, _ptr(perm),
                                  _ptr(offsets), _ptr(ws), nb.value, _stream(stream, cell.device)), "mcc_bin_weighted")
    return perm, offsets


def mcc_bin_static(cell: torch.Tensor, species: torch.Tensor, n_cells: int, n_species: int, perm=None,
                   offsets=None, stream=None):
    """Allocation-free cell sort (library-held counters, no context, no workspace); outputs as mcc_bin. The output
    tensors may be passed in, so that the call itself allocates nothing."""
    n = cell.numel()
    if perm is None:
        perm = torch.empty(n, dtype=torch.int32, device=cell.device)
    if offsets is None:
        offsets = torch.empty(n_cells * n_species + 1, dtype=torch.int64, device=cell.device)
    with torch.cuda.device(cell.device):  # the library's counters are addressed on the current device
        _check(lib().mcc_bin_static(_ptr(cell), _ptr(species), n, n_cells, n_species, _ptr(perm), _ptr(offsets),
                                    _stream(stream, cell.device)), "mcc_bin_static")
    return perm, offsets


def mcc_species_moments(vx, vy, vz, w, offsets, n_cells: int, n_species: int, species, relativistic: bool = False,
                        c: float = 1.0, fail_count=None, out=None, stream=None) -> torch.Tensor:
    """Per-species (sum w, sum m w v (3), kinetic energy, count) and the total of fail_count, as a float64 device
    tensor of 6 n_species + 1 entries (see include/mcc.h)."""
    ctx = context(vx.device)
    P = _particles(vx, vy, vz, w)
    if out is None:
        out = torch.empty(6 * n_species + 1, dtype=torch.float64, device=vx.device)
    _check(lib().mcc_species_moments(ctx.handle, C.byref(P), _ptr(offsets), int(n_cells), int(n_species),
                                     _species(species), int(bool(relativistic)), float(c), _ptr(fail_count),
                                     _ptr(out), _stream(stream, vx.device)), "mcc_species_moments")
    return out


def mcc_gather(x: torch.Tensor, perm: torch.Tensor, stream=None) -> torch.Tensor:
    out = torch.empty_like(x)
    _check(lib().mcc_gather(_ptr(x), _ptr(perm), x.numel(), x.element_size(), _ptr(out),
                            _stream(stream, x.device)), "mcc_gather")
    return out


def mcc_gather_n(xs, perm: torch.Tensor, outs=None, stream=None):
    """One pass over perm for up to 8 arrays: outs[a][k] = xs[a][perm[k]]. Returns the outputs (allocated if not
    given)."""
    xs = list(xs)
    if outs is None:
        outs = [torch.empty_like(x) for x in xs]
    n = perm.numel()
    for x, o in zip(xs, outs):
        if x.numel() != n or o.numel() != n or x.element_size() != o.element_size() or not x.is_contiguous() \
                or not o.is_contiguous():
            raise ValueError("every array and output must be contiguous with one element per permutation entry")
    k = len(xs)
    ins = (C.c_void_p * k)(*[x.data_ptr() for x in xs])
    ous = (C.c_void_p * k)(*[o.data_ptr() for o in outs])
    eb = (C.c_int32 * k)(*[x.element_size() for x in xs])
    _check(lib().mcc_gather_n(ins, ous, eb, k, _ptr(perm), n, _stream(stream, perm.device)), "mcc_gather_n")
    return outs


def mcc_push(x, y, z, vx, vy, vz, grid, dt: float, relativistic: bool = False, c: float = 1.0, cell=None,
             stream=None) -> torch.Tensor:
    """Free-streaming push in a periodic box, positions updated in place (same dtype as the velocities); returns the
    new cell ids (int32). ``grid`` = ((nx, ny, nz), (lx, ly, lz))."""
    (nx, ny, nz), (lx, ly, lz) = grid
    for t in (x, y, z):
        if t.dtype != vx.dtype or not t.is_cuda or not t.is_contiguous() or t.numel() != vx.numel():
            raise TypeError("positions must be contiguous CUDA tensors of the velocities' dtype and length")
    if vx.dtype not in (torch.float64, torch.float32):
        raise TypeError("velocities must be float64 or float32")
    for t in (vx, vy, vz):
        if t.dtype != vx.dtype or not t.is_cuda or not t.is_contiguous() or t.numel() != vx.numel():
            raise TypeError("vx, vy, vz must be contiguous CUDA tensors of one dtype and length")
    P = _Particles(vx.data_ptr(), vy.data_ptr(), vz.data_ptr(), None, vx.numel(),
                   F64 if vx.dtype == torch.float64 else F32_MIXED)  # the push reads no weights
    if cell is None:
        cell = torch.empty(vx.numel(), dtype=torch.int32, device=vx.device)
    g = _Grid(int(nx), int(ny), int(nz), float(lx), float(ly), float(lz))
    _check(lib().mcc_push(C.byref(P), _ptr(x), _ptr(y), _ptr(z), C.byref(g), float(dt), int(bool(relativistic)),
                          float(c), _ptr(cell), _stream(stream, vx.device)), "mcc_push")
    return cell


def mcc_pair(offsets: torch.Tensor, n_cells: int, n_species: int, sa: int, sb: int, inter: int, seed: int,
             step: int, stream=None):
    """Takizuka-Abe pairs of interaction (sa, sb); returns (pair_i, pair_j, flags), each of length N."""
    ctx = context(offsets.device)
    N = int(offsets[-1].item())
    pi = torch.full((max(N, 1),), -1, dtype=torch.int32, device=offsets.device)
    pj = torch.full((max(N, 1),), -1, dtype=torch.int32, device=offsets.device)
    fl = torch.zeros(max(N, 1), dtype=torch.uint8, device=offsets.device)
    _check(lib().mcc_pair(ctx.handle, _ptr(offsets), n_cells, n_species, sa, sb, inter, seed & (2**64 - 1),
                          step & (2**64 - 1), _ptr(pi), _ptr(pj), _ptr(fl), _stream(stream, offsets.device)),
           "mcc_pair")
    return pi[:N], pj[:N], fl[:N]


def mcc_scatter(vx, vy, vz, w, offsets, n_cells, n_species, species, lnL, sa, sb, inter, pairs, params: Params,
                stream=None) -> torch.Tensor:
    """Pair loop of interaction (sa, sb) in place; returns the pre-scatter copy (3, N)."""
    ctx = context(vx.device)
    P = _particles(vx, vy, vz, w)
    backup = torch.empty((3, max(vx.numel(), 1)), dtype=vx.dtype, device=vx.device)
    pi, pj, fl = pairs
    cp = params._c()
    _check(lib().mcc_scatter(ctx.handle, C.byref(P), _ptr(offsets), n_cells, n_species, _species(species),
                             _lnL(lnL, n_species), sa, sb, inter, _ptr(pi), _ptr(pj), _ptr(fl), C.byref(cp),
                             _ptr(backup), _stream(stream, vx.device)), "mcc_scatter")
    return backup[:, : vx.numel()]


ADJOINT_RECOMPUTE, ADJOINT_RECORD, ADJOINT_REPLAY = 0, 1, 2


def adjoint_tape_bytes(device, n_cells: int, max_cell: int, max_corr_passes: int) -> int:
    """Bytes of one recorded adjoint tape (one interaction, every cell)."""
    nb = C.c_size_t()
    _check(lib().mcc_adjoint_tape_size(context(device).handle, int(n_cells), int(max_cell), int(max_corr_passes),
                                       C.byref(nb)), "mcc_adjoint_tape_size")
    return nb.value


def mcc_adjoint(vx, vy, vz, w, offsets, n_cells, n_species, species, lnL, sa, sb, inter, params: Params,
                max_cell: int, out=None, grad=None, gw=None, glnL=None, tape: int = ADJOINT_RECOMPUTE,
                tape_buffer=None, stream=None):
    """One interaction from the state (vx, vy, vz) before it: writes the state after it into ``out`` (three tensors)
    and/or maps ``grad`` (three tensors, dL/dv after, in place) to dL/dv before, adding dL/dw into ``gw`` and
    dL/dlnL_ab into ``glnL`` (one-element float64 tensor). FP64, non-relativistic. With tape = ADJOINT_RECORD the
    call keeps the interaction's tape in ``tape_buffer`` (a uint8 device tensor of adjoint_tape_bytes); a later call
    with tape = ADJOINT_REPLAY on the same interaction runs only the reverse sweep from it."""
    ctx = context(vx.device)
    P = _particles(vx, vy, vz, w)
    if tape == ADJOINT_RECOMPUTE:
        nb = C.c_size_t()
        _check(lib().mcc_adjoint_workspace_size(ctx.handle, int(n_cells), int(max_cell), int(params.max_corr_passes),
                                                C.byref(nb)), "mcc_adjoint_workspace_size")
        ws, nbytes = ctx.workspace("adjoint", nb.value), nb.value
    else:
        if tape_buffer is None or tape_buffer.dtype != torch.uint8 or tape_buffer.device != vx.device:
            raise TypeError("a recorded tape lives in a uint8 tensor on the particles' device")
        ws, nbytes = tape_buffer, tape_buffer.numel()
    o = out if out is not None else (None, None, None)
    g = grad if grad is not None else (None, None, None)
    for t in [*(x for x in o if x is not None), *(x for x in g if x is not None), gw, glnL]:
        if t is not None and (t.dtype != torch.float64 or not t.is_contiguous() or t.device != vx.device):
            raise TypeError("outputs and gradients must be contiguous float64 tensors on the particles' device")
    cp = params._c()
    _check(lib().mcc_adjoint(ctx.handle, C.byref(P), _ptr(offsets), n_cells, n_species, _species(species),
                             _lnL(lnL, n_species), sa, sb, inter, C.byref(cp), int(max_cell), _ptr(o[0]), _ptr(o[1]),
                             _ptr(o[2]), _ptr(g[0]), _ptr(g[1]), _ptr(g[2]), _ptr(gw), _ptr(glnL), int(tape),
                             _ptr(ws), nbytes, _stream(stream, vx.device)), "mcc_adjoint")


def mcc_correct(vx, vy, vz, w, offsets, n_cells, n_species, species, sa, sb, inter, params: Params,
                backup: torch.Tensor, stream=None):
    """Moment correction of interaction (sa, sb) in place; returns (corr_pairs, fail_flags) per cell."""
    ctx = context(vx.device)
    P = _particles(vx, vy, vz, w)
    bk = backup.contiguous()
    if bk.dim() != 2 or bk.shape[0] != 3 or bk.dtype != vx.dtype:
        raise TypeError("backup must be the (3, N) tensor returned by mcc_scatter")
    corr = torch.zeros(max(n_cells, 1), dtype=torch.int32, device=vx.device)
    fail = torch.zeros(max(n_cells, 1), dtype=torch.int32, device=vx.device)
    cp = params._c()
    _check(lib().mcc_correct(ctx.handle, C.byref(P), _ptr(offsets), n_cells, n_species, _species(species), sa, sb,
                             inter, C.byref(cp), _ptr(bk), _ptr(corr), _ptr(fail), _stream(stream, vx.device)),
           "mcc_correct")
    return corr[:n_cells], fail[:n_cells]


def default_interactions(n_species: int):
    return [(a, b) for a in range(n_species) for b in range(a, n_species)]


def mcc_step_fused(vx, vy, vz, w, offsets, n_cells, n_species, species, lnL, params: Params, n_steps: int = 1,
                   max_cell: int | None = None, interactions=None, corr_pairs=None, fail_count=None, stream=None):
    """n_steps whole collision steps in place (one persistent kernel launch per step). Returns the per-cell
    accumulated (corr_pairs, fail_count) tensors."""
    ctx = context(vx.device)
    P = _particles(vx, vy, vz, w)
    inter = default_interactions(n_species) if interactions is None else [tuple(x) for x in interactions]
    flat = (C.c_int32 * (2 * len(inter)))(*[int(v) for ab in inter for v in ab])
    if max_cell is None:
        max_cell = int((offsets[n_species::n_species] - offsets[:-1:n_species]).max().item()) if n_cells else 0
    if corr_pairs is None:
        corr_pairs = torch.zeros(max(n_cells, 1), dtype=torch.int32, device=vx.device)
    if fail_count is None:
        fail_count = torch.zeros(max(n_cells, 1), dtype=torch.int32, device=vx.device)
    nb = C.c_size_t()
    _check(lib().mcc_step_workspace_size(ctx.handle, P.prec, int(n_cells), int(max_cell), C.byref(nb)),
           "mcc_step_workspace_size")
    ws = ctx.workspace(("step", P.prec), nb.value)
    cp = params._c()
    _check(lib().mcc_step_fused(ctx.handle, C.byref(P), _ptr(offsets), n_cells, n_species, _species(species),
                                _lnL(lnL, n_species), flat, len(inter), C.byref(cp), int(n_steps), int(max_cell),
                                _ptr(corr_pairs), _ptr(fail_count), _ptr(ws), nb.value,
                                _stream(stream, vx.device)), "mcc_step_fused")
    return corr_pairs[:n_cells], fail_count[:n_cells]


def sync_status(device=None, stream=None):
    """Synchronise and raise MccError if the device latched an error since the last check."""
    ctx = context(device)
    rc = ctx.sync_status(stream)
    _check(rc, "device status")
