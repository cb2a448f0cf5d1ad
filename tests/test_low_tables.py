"""Host-side check of the low-diagonal kernel's tables and programs (no GPU):
bounds of every shared-memory index, and bit-exact agreement of the
table-driven program with a plain recursive W-cycle (tests/low_tables_check.cu)."""
import os
import shutil
import subprocess

import pytest

from paper_1907_12334_gb300 import build

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_1907_12334_gb300", "csrc")


def test_low_tables_bounds_and_program(tmp_path):
    nvcc = build.nvcc()
    if not shutil.which(nvcc) and not os.path.exists(nvcc):
        pytest.skip("nvcc not found")
    exe = tmp_path / "low_tables_check"
    cmd = [nvcc, *build.ARCH, "-std=c++17", "--expt-relaxed-constexpr", "-I", build.INCLUDE, "-I", CSRC,
           os.path.join(HERE, "low_tables_check.cu"), os.path.join(CSRC, "api.cu"), "-o", str(exe)]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-2000:]
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout[-2000:]
    assert "0 out of range" in r.stdout and " 0 differ" in r.stdout
