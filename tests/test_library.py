"""CPU-side checks of the C-ABI library: it builds for sm_103a, loads, and exports
every entry point include/dualpf.h declares (no compute calls without a GPU)."""
import os
import re
import subprocess

import pytest

from paper_2111_04577_gb300 import build, binding

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    src = open(os.path.join(ROOT, "include", "dualpf.h")).read()
    return sorted(set(re.findall(r"\b(pf_[a-z_]+)\s*\(", src)))


def test_builds_and_exports_every_declared_symbol():
    lib = build.build()
    out = subprocess.run(["nm", "-D", "--defined-only", lib], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (pf_[a-z_]+)\b", out))
    declared = header_functions()
    assert declared, "no declarations found"
    missing = [f for f in declared if f not in exported]
    assert not missing, missing
    assert set(binding.EXPORTS) <= exported


def test_loads_and_reports_errors_without_a_gpu():
    build.build()
    lib = binding.load()
    import ctypes as C
    h = C.c_void_p()
    # a non-cubic grid is rejected before any device work
    gd = binding.GridDesc(8, 1, 4, 1.0, 0.125, 3.0, binding.PF_FP64, 1)
    rc = lib.pf_init_grid(C.byref(h), C.byref(gd), None)
    assert rc == -1
    assert b"cube" in lib.pf_last_error(None)
    gd = binding.GridDesc(22, 1, 4, 22.0, 1.0, 4.0, binding.PF_FP64, 1)  # 11 is not 2^a3^b5^c7^d
    assert lib.pf_init_grid(C.byref(h), C.byref(gd), None) == -3
