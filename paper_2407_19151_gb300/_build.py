"""In-tree build of the CUDA library (nvcc, sm_103a only) into ``paper_2407_19151_gb300/_build``."""
from __future__ import annotations

import os
import platform
import subprocess
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
SOURCES = ["mcc_abi.cu", "mcc_cell.cu", "mcc_bin.cu", "mcc_adjoint.cu", "mcc_pic.cu", "mcc_group_f32.cu",
           "mcc_group_f32rel.cu", "mcc_moments.cu"]
HEADERS = ["mcc_device.cuh", "mcc_kernels.h", "mcc_pic.h", "mcc_group.cuh"]
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc" if os.path.exists("/usr/local/cuda/bin/nvcc") else "nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", os.path.join(ROOT, "include")]
EXTRA = os.environ.get("MCC_NVCC_FLAGS", "").split()
# The mixed-precision group kernels take float division and square root from the hardware approximations (about
# 2 ulp), like the explicit fast intrinsics of their pair kinematics; every other unit keeps IEEE float division.
UNIT_FLAGS = {"mcc_group_f32.cu": ["-prec-div=false", "-prec-sqrt=false"],
              "mcc_group_f32rel.cu": ["-prec-div=false", "-prec-sqrt=false"]}


def lib_path(debug_bounds: bool = False, phase_clocks: bool = False) -> str:
    tag = ("_bounds" if debug_bounds else "") + ("_clocks" if phase_clocks else "")
    return os.path.join(BUILD, f"libmcc{tag}.{platform.machine()}.so")


def source_hash() -> str:
    """Hash of every source the library is built from (keys the autotuner's cache and the profile records)."""
    import hashlib
    h = hashlib.sha256()
    for f in [os.path.join(CSRC, f) for f in SOURCES + HEADERS] + [os.path.join(ROOT, "include", "mcc.h")]:
        with open(f, "rb") as fh:
            h.update(fh.read())
    h.update(repr(sorted(UNIT_FLAGS.items())).encode())
    return h.hexdigest()[:16]


def _newest_input() -> float:
    files = [os.path.join(CSRC, f) for f in SOURCES + HEADERS] + [os.path.join(ROOT, "include", "mcc.h"),
                                                                 os.path.abspath(__file__)]
    return max(os.path.getmtime(f) for f in files)


def build(force: bool = False, verbose: bool = False, out: str | None = None, debug_bounds: bool = False,
          phase_clocks: bool = False) -> str:
    """Compile every translation unit in parallel, link the shared library; skip if up to date. debug_bounds builds
    the bounds-checked variant (-DMCC_DEBUG_BOUNDS), phase_clocks the phase-timing variant (-DMCC_PHASE_CLOCKS),
    each into its own file."""
    out = out or lib_path(debug_bounds, phase_clocks)
    extra = EXTRA + (["-DMCC_DEBUG_BOUNDS"] if debug_bounds else []) + (["-DMCC_PHASE_CLOCKS"] if phase_clocks else [])
    if not force and os.path.exists(out) and os.path.getmtime(out) >= _newest_input():
        return out
    os.makedirs(os.path.dirname(out), exist_ok=True)

    def compile_one(src: str) -> str:
        obj = os.path.join(os.path.dirname(out), f"{os.path.splitext(src)[0]}.{os.path.basename(out)}.o")
        cmd = [NVCC, *ARCH, *FLAGS, *UNIT_FLAGS.get(src, []), *extra, "-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
        if verbose and r.stderr:
            print(r.stderr)
        return obj

    with ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = out + f".tmp{os.getpid()}"
    r = subprocess.run([NVCC, *ARCH, "-shared", "-o", tmp, *objs], capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, out)
    return out


if __name__ == "__main__":
    print(build(force=True, verbose=True))
