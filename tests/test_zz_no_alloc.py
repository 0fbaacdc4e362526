"""The allocation-free sweep entry point against the regular one.

jac_sweep_noalloc serves callers that cannot allocate device memory when they
need a solve (a memory pool that owns the device, loops that must not stall on
cudaMalloc's device synchronisation, hosts that forbid allocation after
start-up): it works on the caller's buffers and a fixed scratch area compiled
into the library.  These tests call it through the C ABI and compare it with
jac_setup + jac_sweep on the same inputs, on calls made back to back (the
scratch area keeps the previous call's contents).  This file is collected
last so that a run stopping at the first failure has run every other test.
"""
import ctypes

import numpy as np
import pytest

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


def _relres_tol(A, b, x):
    bn = np.linalg.norm(b)
    return RTOL * (bn + np.linalg.norm(abs(A.scipy()) @ np.abs(x))) / bn


def _regular(A, b, x0, k):
    ctx = J.jac_setup(A, b, J.JAC_BANDROW, 3, J.opts(variant=2))
    try:
        J.jac_set_x(ctx, x0)
        rel = J.jac_sweep(ctx, k)
        return J.jac_get_x(ctx), rel
    finally:
        J.jac_free(ctx)


def _cases():
    A = W.laplace7(16)
    yield "lap7_16", A, W.solution_and_rhs(A, 0)[1]
    A = W.fe27_deleted(10, seed=3)
    yield "fe27", A, W.solution_and_rhs(A, 1)[1]
    A = W.diffusion7((13, 11, 7), seed=2)
    yield "ragged", A, W.solution_and_rhs(A, 4)[1]


@pytest.mark.parametrize("name,A,b", list(_cases()))
def test_noalloc_matches_regular_entry_point_on_consecutive_calls(name, A, b):
    import torch
    rng = np.random.default_rng(7)
    x0 = rng.uniform(-1, 1, A.n)
    rp, cl, vl, db = _dev(A.rowptr), _dev(A.col), _dev(A.val), _dev(b)
    xin = _dev(x0)
    outs = [torch.empty(A.n, dtype=torch.float64, device="cuda") for _ in range(3)]
    x = x0
    # two single-sweep calls in a row, each against the regular path fed the same input
    for call in range(2):
        rel = J.jac_sweep_noalloc(rp, cl, vl, db, xin, outs[call], 1)
        got = outs[call].cpu().numpy()
        ref, rref = _regular(A, b, x, 1)
        err = np.abs(got - ref)
        assert np.all(err <= RTOL * _scale(A, b, x) + 1e-300), (call, err.max())
        assert abs(rel - rref) <= _relres_tol(A, b, x)
        x = got
        xin = outs[call]
    # a longer call after them: same iterate and residual as 25 regular sweeps
    rel = J.jac_sweep_noalloc(rp, cl, vl, db, xin, outs[2], 25)
    ref, rref = _regular(A, b, x, 25)
    got = outs[2].cpu().numpy()
    assert np.linalg.norm(got - ref) <= 1e-12 * np.linalg.norm(ref)
    assert abs(rel - rref) <= 1e-12


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
    ref, rref = _regular(A, b, np.zeros(A.n), 3)
    assert np.linalg.norm(out.cpu().numpy() - ref) <= 1e-13 * np.linalg.norm(ref)
    assert abs(rel - rref) <= 1e-13
