"""GB300-native (sm_103a) weighted, moment-preserving Monte-Carlo Coulomb collision step.

The collision step of Angus et al., "Moment-preserving Monte-Carlo Coulomb collision method for particle codes":
cell binning, Takizuka-Abe random pairing, TA77 / N97 scattering generalised to weighted particles, and the
post-scatter moment correction that restores exact momentum and energy conservation (non-relativistic and
relativistic). The work runs in hand-written CUDA kernels behind the C ABI of ``include/mcc.h``; this package is
the thin Python binding (same names as the C entry points) plus the seeded synthetic workloads.
"""
from ._build import build as _build_library, lib_path
from .adjoint import collision_steps
from .autotune import autotune
from .pic import PicLoop
from ._binding import (ADJOINT_RECOMPUTE, ADJOINT_RECORD, ADJOINT_REPLAY, F32_MIXED, F64, FAIL_ERROR,
                       FAIL_MOMENTUM_ONLY, FAIL_ROLLBACK, GROUP_CLASSES, N97, TA77, Context, MccError, Params,
                       adjoint_tape_bytes, context, default_interactions, lib, mcc_adjoint, mcc_bin, mcc_bin_static,
                       mcc_bin_weighted, mcc_correct, mcc_gather, mcc_gather_n, mcc_pair, mcc_push, mcc_scatter,
                       mcc_species_moments, mcc_step_fused, sync_status)


def build(force: bool = False) -> str:
    """Compile the CUDA library for sm_103a (in tree) and return its path."""
    return _build_library(force=force)


__all__ = [
    "build", "lib_path", "lib", "context", "Context", "Params", "MccError", "mcc_bin", "mcc_bin_static",
    "mcc_bin_weighted", "mcc_gather", "mcc_gather_n", "mcc_push", "PicLoop", "mcc_adjoint", "collision_steps", "mcc_pair",
    "mcc_scatter", "mcc_correct", "mcc_species_moments", "mcc_step_fused", "sync_status", "default_interactions", "TA77", "N97", "F64",
    "F32_MIXED", "GROUP_CLASSES", "ADJOINT_RECOMPUTE", "ADJOINT_RECORD", "ADJOINT_REPLAY", "adjoint_tape_bytes", "FAIL_ROLLBACK", "FAIL_MOMENTUM_ONLY", "FAIL_ERROR", "autotune",
]
