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
    assert L.gfp_create_grid(8, 1536, 8, 1.0, None, ctypes.byref(h)) == -2   # 2^9 3, above the 1024 limit
    assert L.gfp_create_grid(8, 8, 2048, 1.0, None, ctypes.byref(h)) == -2
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


def test_struct_layouts_match_the_header(tmp_path):
    """The binding's ctypes mirrors of gfp_scheme and gfp_result have the header's size and field
    offsets (compiled with the host C compiler)."""
    import ctypes
    import shutil
    from paper_2009_03762_gb300 import gfp
    cc = shutil.which("gcc") or shutil.which("cc")
    if not cc:
        pytest.skip("no C compiler")
    res_fields = [f[0] for f in gfp._Result._fields_]
    sch_fields = [f[0] for f in gfp.Scheme._fields_]
    # same member names, in order, as the header's typedefs (a trailing int could hide in padding)
    hdr = open(os.path.join(ROOT, "include", "gfp.h")).read()
    for name, fields in (("gfp_result", res_fields), ("gfp_scheme", sch_fields)):
        body = re.search(r"typedef struct \{([^{}]*)\}\s*%s;" % name, hdr).group(1)
        body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
        members = re.findall(r"(\w+)\s*(?:\[\d+\])?\s*;", body)
        assert members == fields, (name, members, fields)
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "gfp.h"', "int main(void) {",
             '  printf("gfp_result %zu\\n", sizeof(gfp_result));', '  printf("gfp_scheme %zu\\n", sizeof(gfp_scheme));']
    lines += ['  printf("r.%s %%zu\\n", offsetof(gfp_result, %s));' % (f, f) for f in res_fields]
    lines += ['  printf("s.%s %%zu\\n", offsetof(gfp_scheme, %s));' % (f, f) for f in sch_fields]
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = dict(l.split() for l in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.splitlines())
    assert int(out["gfp_result"]) == ctypes.sizeof(gfp._Result)
    assert int(out["gfp_scheme"]) == ctypes.sizeof(gfp.Scheme)
    for f in res_fields:
        assert int(out["r." + f]) == getattr(gfp._Result, f).offset, f
    for f in sch_fields:
        assert int(out["s." + f]) == getattr(gfp.Scheme, f).offset, f
