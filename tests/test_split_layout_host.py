"""Host logic of the split interface layout and of the tiler's warp
alignment, checked without a GPU: tests/cpp/split_layout_check.cpp is built
with the library's host partitioner source and run."""
import os
import shutil
import subprocess

import pytest

from conftest import ROOT


def test_split_layout_invariants(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    csrc = os.path.join(ROOT, "paper_2112_02377_gb300", "csrc")
    exe = os.path.join(str(tmp_path), "split_layout_check")
    subprocess.check_call([cxx, "-std=c++17", "-O2", "-Wall", "-Wextra", "-Werror", "-I", csrc,
                           os.path.join(ROOT, "tests", "cpp", "split_layout_check.cpp"),
                           os.path.join(csrc, "jac_partition.cpp"), "-o", exe])
    out = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert out.returncode == 0 and out.stdout.strip().endswith("ok"), out.stdout + out.stderr
