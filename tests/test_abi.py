"""CPU checks of the C ABI library: it builds, loads, and exports every symbol include/gfp.h declares."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            names += re.findall(r"^\s*(?:int|const char\*)\s+(gfp_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def libpath():
    from paper_2009_03762_gb300 import _build
    if not os.path.exists(_build.LIB):
        _build.build()
    return _build.LIB


def test_header_declares_entry_points():
    names = _declared()
    for n in ("gfp_create_grid", "gfp_set_phases", "gfp_solve", "gfp_effective_stiffness", "gfp_grad",
              "gfp_destroy_grid", "gfp_error_string"):
        assert n in names


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.check_output(["nm", "-D", "--defined-only", libpath]).decode()
    exported = set(re.findall(r"\bT\s+(gfp_\w+)", out))
    missing = [n for n in _declared() if n not in exported]
    assert not missing, missing


def test_library_loads_and_reports_errors_without_gpu(libpath):
    import ctypes
    from paper_2009_03762_gb300 import gfp
    L = gfp.lib()
    assert L.gfp_error_string(0) == b"ok"
    assert b"unsupported grid size" in L.gfp_error_string(-2)
    # argument validation happens before any device call
    h = ctypes.c_void_p()
    assert L.gfp_create_grid(5, 8, 8, 1.0, None, ctypes.byref(h)) == -2
    assert L.gfp_create_grid(0, 8, 8, 1.0, None, ctypes.byref(h)) == -1
    assert L.gfp_create_grid(8, 8, 8, -1.0, None, ctypes.byref(h)) == -1


def test_product_package_does_not_import_the_oracle():
    pkg = os.path.join(ROOT, "paper_2009_03762_gb300")
    bad = re.compile(r"^\s*(from|import)\s+oracle\b|gfp_oracle|[\'\"]oracle[/\'\"]", re.M)
    for dirpath, _, files in os.walk(pkg):
        for fn in files:
            if fn.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                src = open(os.path.join(dirpath, fn)).read()
                assert not bad.search(src), fn
