"""Register budgets of the FP32 256^3 hot kernels, from ptxas's report of a build for sm_103a.

Their occupancy rests on these numbers (ten 96-thread x-pass CTAs per SM at 64 registers; two
384-thread z-pass CTAs at 80): FP64-only branches once doubled the x-pass's registers unnoticed."""
import os
import re
import shutil
import subprocess
import tempfile

import pytest

pytestmark = pytest.mark.slow

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2009_03762_gb300", "csrc")


def _nvcc():
    home = os.environ.get("CUDA_HOME", "/usr/local/cuda")
    cand = os.path.join(home, "bin", "nvcc")
    return cand if os.path.exists(cand) else shutil.which("nvcc")


def _ptxas_report():
    nvcc = _nvcc()
    if not nvcc:
        pytest.skip("nvcc not found")
    with tempfile.TemporaryDirectory() as tmp:
        out = subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17",
                              "-Xcompiler", "-fPIC", "-Xptxas", "-v", "-c", os.path.join(CSRC, "gfp_k32.cu"),
                              "-o", os.path.join(tmp, "k32.o")], capture_output=True, text=True)
    assert out.returncode == 0, out.stderr[-2000:]
    report = {}
    name = None
    for line in out.stderr.splitlines():
        m = re.search(r"Compiling entry function '(\S+)'", line)
        if m:
            name = m.group(1)
            continue
        m = re.search(r"(\d+) bytes spill stores", line)
        if m and name:
            report.setdefault(name, {})["spill"] = int(m.group(1))
        m = re.search(r"Used (\d+) registers", line)
        if m and name:
            report.setdefault(name, {})["regs"] = int(m.group(1))
    return report


def test_fp32_hot_kernel_register_budgets():
    rep = _ptxas_report()
    x = [v for k, v in rep.items() if k.startswith("_ZN3gfp15pass_x_c_kernelIfLi256EE")]
    z = [v for k, v in rep.items() if k.startswith("_ZN3gfp16pass_z_c2_kernelIfLi256EE")]
    assert len(x) == 1 and len(z) == 1, sorted(rep)[:10]
    assert x[0]["regs"] <= 64 and x[0].get("spill", 0) == 0, x
    assert z[0]["regs"] <= 80 and z[0].get("spill", 0) <= 16, z
