"""Host logic of the split interface layout and of the tiler's warp
alignment, checked without a GPU: tests/cpp/split_layout_check.cpp is built
with the library's host partitioner source and run, once optimised and once
under gcc's AddressSanitizer and UndefinedBehaviorSanitizer (out-of-bounds
accesses, leaks, signed overflow and other undefined behaviour in the
partitioner abort the run)."""
import os
import shutil
import subprocess

import pytest

from conftest import ROOT

SANITIZE = ["-O1", "-g", "-fno-omit-frame-pointer", "-fsanitize=address,undefined", "-fno-sanitize-recover=all"]


def _sanitizers_available(cxx, tmp_path) -> bool:
    src = os.path.join(tmp_path, "probe.cpp")
    with open(src, "w") as f:
        f.write("int main() { return 0; }\n")
    res = subprocess.run([cxx, *SANITIZE, src, "-o", os.path.join(tmp_path, "probe")], capture_output=True)
    return res.returncode == 0


@pytest.mark.parametrize("mode", ["optimised", "sanitized"])
def test_split_layout_invariants(tmp_path, mode):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    flags = ["-O2"]
    env = dict(os.environ)
    if mode == "sanitized":
        if not _sanitizers_available(cxx, str(tmp_path)):
            pytest.skip("the compiler has no AddressSanitizer / UndefinedBehaviorSanitizer runtime")
        flags = SANITIZE
        env.update(ASAN_OPTIONS="detect_leaks=1:halt_on_error=1", UBSAN_OPTIONS="print_stacktrace=1")
    csrc = os.path.join(ROOT, "paper_2112_02377_gb300", "csrc")
    exe = os.path.join(str(tmp_path), "split_layout_check")
    subprocess.check_call([cxx, "-std=c++17", *flags, "-Wall", "-Wextra", "-Werror", "-I", csrc,
                           os.path.join(ROOT, "tests", "cpp", "split_layout_check.cpp"),
                           os.path.join(csrc, "jac_partition.cpp"), "-o", exe])
    out = subprocess.run([exe], capture_output=True, text=True, timeout=300, env=env)
    assert out.returncode == 0 and out.stdout.strip().endswith("ok"), out.stdout + out.stderr
