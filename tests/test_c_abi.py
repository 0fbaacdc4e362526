"""The C ABI from plain C: tests/c/solve_laplace7.c compiled as C99 against
include/jacobi.h and linked with libjacobi_gb300.so."""
import os
import re
import shutil
import subprocess

import numpy as np
import pytest

from conftest import ROOT
from oracle import oracle as O
from paper_2112_02377_gb300 import _build
from paper_2112_02377_gb300 import workloads as W


def _compile(tmp_path):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    _build.build()
    exe = os.path.join(tmp_path, "solve_laplace7")
    libdir = os.path.dirname(_build.LIB)
    subprocess.check_call([cc, "-std=c99", "-O2", "-Wall", "-Wextra", "-Werror", "-pedantic",
                           "-I", os.path.join(ROOT, "include"), os.path.join(ROOT, "tests", "c", "solve_laplace7.c"),
                           "-o", exe, "-L", libdir, "-ljacobi_gb300", "-Wl,-rpath," + libdir, "-lm"])
    return exe


def test_c_program_builds_and_fails_cleanly_without_a_gpu(tmp_path):
    import torch
    exe = _compile(str(tmp_path))
    if torch.cuda.is_available():
        pytest.skip("a GPU is present (see the gpu test)")
    out = subprocess.run([exe, "8"], capture_output=True, text=True, timeout=120)
    assert out.returncode == 3, out.stdout + out.stderr        # JAC_ECUDA
    assert out.stdout.startswith("jac_setup: ")


@pytest.mark.gpu
def test_c_program_solves_like_the_oracle(tmp_path):
    exe = _compile(str(tmp_path))
    m = 12
    out = subprocess.run([exe, str(m)], capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stdout + out.stderr
    got = dict(re.findall(r"(\w+)=(\S+)", out.stdout))
    A = W.laplace7(m)
    b = A.scipy() @ np.ones(A.n)
    _, k, rel, st = O.solve(A, b, None, tol=1e-8, maxit=100000)
    assert int(got["sweeps"]) == k
    assert abs(float(got["relres"]) - rel) <= 1e-12 * (1 + rel) + 1e-14
    assert float(got["maxerr"]) <= 1e-6
