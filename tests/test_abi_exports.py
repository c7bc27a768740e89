"""The C-ABI library loads on the host and exports every entry point declared in include/mcc.h (CPU only, no compute
call is made)."""
import ctypes
import os
import re

import paper_2407_19151_gb300 as mcc

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    text = open(os.path.join(ROOT, "include", "mcc.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[\w\*\s]+?\b(mcc_\w+)\s*\(", text, flags=re.M)))


def test_header_declares_the_calls():
    names = declared_functions()
    for required in ["mcc_bin", "mcc_pair", "mcc_scatter", "mcc_correct", "mcc_step_fused", "mcc_create",
                     "mcc_destroy", "mcc_sync_status", "mcc_status_string"]:
        assert required in names


def test_library_exports_every_declared_symbol():
    path = mcc.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_status_strings_without_gpu():
    lib = mcc.lib()
    assert lib.mcc_status_string(0) == b"ok"
    assert b"energy correction" in lib.mcc_status_string(-5)
