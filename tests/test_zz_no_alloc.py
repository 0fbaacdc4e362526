"""The allocation-free sweep entry point against the oracle.

jac_sweep_noalloc serves callers that cannot allocate device memory when they
need a solve (a memory pool that owns the device, loops that must not stall on
cudaMalloc's device synchronisation, hosts that forbid allocation after
start-up): it works on the caller's buffers and a fixed scratch area compiled
into the library.  These tests call it through the C ABI on calls made back to
back (the scratch area keeps the previous call's contents) and compare every
result with the CPU oracle's sweep on the same input, element by element.
This file is collected last so that a run stopping at the first failure has
run every other test.

Tolerances.  One sweep from the same input: |x_gpu - x_oracle|_i <=
1e-13 * scale_i with scale_i = (|b_i| + sum_{j != i} |a_ij x_j|) / |a_ii|, the
per-sweep bar of the other parity tests.  After k sweeps from the same input
the two runs' differences pass through the iteration matrix T = -D^{-1}(L+U);
every operator here has ||T||_inf <= 1 (checked), so each sweep adds at most
one rounding difference of each side and the difference stays below
2 k 1e-13 max_m ||scale(x_m)||_inf in every component.
"""
import ctypes

import numpy as np
import pytest

from oracle import oracle as O
from paper_2112_02377_gb300 import jacobi as J
from paper_2112_02377_gb300 import workloads as W

pytestmark = pytest.mark.gpu

RTOL = 1e-13          # the per-sweep tolerance of tests/test_gpu_parity.py


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _scale(A, b, x):
    S = A.scipy()
    d = S.diagonal()
    off = abs(S) @ np.abs(x) - np.abs(d) * np.abs(x)
    return (np.abs(b) + off) / np.abs(d)


def _relres_tol(A, b, x, err=0.0):
    """Bound on |relres_gpu - relres_oracle| for iterates that differ by at
    most `err` in every component."""
    bn = np.linalg.norm(b)
    absA = abs(A.scipy())
    return (RTOL * (bn + np.linalg.norm(absA @ np.abs(x))) + err * np.linalg.norm(absA @ np.ones(A.n))) / bn


def _t_inf_norm(A):
    S = A.scipy()
    d = np.abs(S.diagonal())
    return float(np.max((abs(S) @ np.ones(A.n) - d) / d))


def _cases():
    A = W.laplace7(16)
    yield "lap7_16", A, W.solution_and_rhs(A, 0)[1]
    A = W.fe27_deleted(10, seed=3)
    yield "fe27", A, W.solution_and_rhs(A, 1)[1]
    A = W.diffusion7((13, 11, 7), seed=2)
    yield "ragged", A, W.solution_and_rhs(A, 4)[1]


@pytest.mark.parametrize("name,A,b", list(_cases()))
def test_noalloc_matches_oracle_on_consecutive_calls(name, A, b):
    import torch
    assert _t_inf_norm(A) <= 1.0 + 1e-15
    Mo = O.prepare(A)
    rng = np.random.default_rng(7)
    x0 = rng.uniform(-1, 1, A.n)
    rp, cl, vl, db = _dev(A.rowptr), _dev(A.col), _dev(A.val), _dev(b)
    xin = _dev(x0)
    outs = [torch.empty(A.n, dtype=torch.float64, device="cuda") for _ in range(3)]
    x = x0
    # two single-sweep calls in a row, each against the oracle's sweep of the same input
    for call in range(2):
        rel = J.jac_sweep_noalloc(rp, cl, vl, db, xin, outs[call], 1)
        got = outs[call].cpu().numpy()
        y, ss, mx = O.sweep(Mo, b, x)
        err = np.abs(got - y)
        sc = _scale(A, b, x)
        assert np.all(err <= RTOL * sc + 1e-300), (call, float(np.max(err / (sc + 1e-300))))
        assert abs(rel - np.sqrt(ss) / np.linalg.norm(b)) <= _relres_tol(A, b, x)
        x = got
        xin = outs[call]
    # a longer call after them: 25 sweeps against 25 oracle sweeps from the same input
    k = 25
    rel = J.jac_sweep_noalloc(rp, cl, vl, db, xin, outs[2], k)
    got = outs[2].cpu().numpy()
    y, maxsc = x, 0.0
    for m in range(k):
        maxsc = max(maxsc, float(_scale(A, b, y).max()))
        prev = y
        y, ss, mx = O.sweep(Mo, b, y)
    bound = 2 * k * RTOL * maxsc
    assert np.all(np.abs(got - y) <= bound), float(np.max(np.abs(got - y)) / bound)
    # the test value is that of x^{k-1}, whose components differ by at most 2 (k-1) 1e-13 maxsc
    assert abs(rel - np.sqrt(ss) / np.linalg.norm(b)) <= _relres_tol(A, b, prev, 2 * (k - 1) * RTOL * maxsc)


def test_noalloc_rejects_bad_arguments():
    import torch
    A = W.laplace7(6)
    xs, b = W.solution_and_rhs(A, 0)
    rp, cl, vl, db = _dev(A.rowptr), _dev(A.col), _dev(A.val), _dev(b)
    x0 = torch.zeros(A.n, dtype=torch.float64, device="cuda")
    out = torch.empty_like(x0)
    L = J.lib()
    P = lambda t: ctypes.c_void_p(t.data_ptr())
    rel = ctypes.c_double()
    # more rows than the fixed scratch area holds: rejected before any pointer is read
    st = L.jac_sweep_noalloc(4194305, P(rp), P(cl), P(vl), P(db), P(x0), P(out), 1, ctypes.byref(rel), None)
    assert st == J.JAC_EINVAL and "scratch limit" in J.jac_last_error()
    st = L.jac_sweep_noalloc(A.n, P(rp), P(cl), P(vl), P(db), P(x0), P(x0), 1, ctypes.byref(rel), None)
    assert st == J.JAC_EINVAL and "alias" in J.jac_last_error()
    st = L.jac_sweep_noalloc(A.n, P(rp), P(cl), P(vl), P(db), P(x0), P(out), -1, ctypes.byref(rel), None)
    assert st == J.JAC_EINVAL
    # a zero diagonal is reported, and the next call still works
    k5 = [e for e in range(A.rowptr[5], A.rowptr[6]) if A.col[e] == 5][0]
    v2 = A.val.copy()
    v2[k5] = 0.0
    with pytest.raises(J.JacobiError) as ei:
        J.jac_sweep_noalloc(rp, cl, _dev(v2), db, x0, out, 3)
    assert ei.value.status == J.JAC_ENUMERIC
    rel = J.jac_sweep_noalloc(rp, cl, vl, db, x0, out, 3)
    Mo = O.prepare(A)
    y, maxsc = np.zeros(A.n), 0.0
    for m in range(3):
        maxsc = max(maxsc, float(_scale(A, b, y).max()))
        prev = y
        y, ss, mx = O.sweep(Mo, b, y)
    assert np.all(np.abs(out.cpu().numpy() - y) <= 2 * 3 * RTOL * maxsc)
    assert abs(rel - np.sqrt(ss) / np.linalg.norm(b)) <= _relres_tol(A, b, prev, 2 * 2 * RTOL * maxsc)
