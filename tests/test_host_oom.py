"""A host allocation that fails inside the library comes back as JAC_ENOMEM
with a message, not as a C++ exception unwinding through the C ABI into the
caller.  The child process lowers its own address-space limit (soft limit
only) just before the call, so the library's first large std::vector fails;
nothing is ever touched beyond the limit, and no GPU is used."""
import os
import subprocess
import sys
import textwrap

import pytest

from conftest import ROOT

CHILD = textwrap.dedent(r"""
    import resource, sys
    sys.path.insert(0, sys.argv[1])
    import numpy as np
    from paper_2112_02377_gb300 import jacobi as J, workloads as W
    J.lib()
    A = W.laplace7(100)                      # 1,000,000 rows, 6,940,000 entries
    def vm_bytes():
        for line in open("/proc/self/status"):
            if line.startswith("VmSize:"):
                return int(line.split()[1]) * 1024
    soft, hard = resource.getrlimit(resource.RLIMIT_AS)
    lim = vm_bytes() + (48 << 20)            # the host copy of A alone needs ~90 MB
    resource.setrlimit(resource.RLIMIT_AS, (lim, hard))
    try:
        J.jac_partition_plan(A, J.JAC_BANDROW, 4, J.opts())
        print("NO-ERROR")
    except J.JacobiError as e:
        print("STATUS", e.status, e)
    resource.setrlimit(resource.RLIMIT_AS, (soft, hard))
    perm, part_ptr = J.jac_partition_plan(A, J.JAC_BANDROW, 4, J.opts())
    print("AFTER", len(perm), [int(v) for v in part_ptr])
""")


@pytest.mark.skipif(not sys.platform.startswith("linux"), reason="needs /proc and RLIMIT_AS")
def test_host_allocation_failure_is_a_status_not_a_crash():
    out = subprocess.run([sys.executable, "-c", CHILD, ROOT], capture_output=True, text=True, timeout=300,
                         env=dict(os.environ, CUDA_VISIBLE_DEVICES=""))
    assert out.returncode == 0, out.stdout + out.stderr
    lines = out.stdout.splitlines()
    status = [l for l in lines if l.startswith("STATUS")]
    assert status, out.stdout
    assert status[0].split()[1] == "2" and "host allocation" in status[0]      # JAC_ENOMEM
    assert "AFTER 1000000 [0, 250000, 500000, 750000, 1000000]" in lines
