"""Batched solves: many independent systems x several right-hand sides in one
persistent launch.  Every (system, right-hand side) must behave exactly like
its own single-system Jacobi run (Sec. 3 iteration, Algorithm 1 test): same
stopping sweep, same iterate, same test value.

Tolerances, element by element for every (system, right-hand side):
* one sweep from the same input: |x_gpu - x_oracle|_i <= 1e-13 * scale_i,
  scale_i = (|b_i| + sum_{j != i} |a_ij x_j|) / |a_ii| (the bar of
  tests/test_gpu_parity.py);
* k sweeps from the same input: every operator here has ||T||_inf <= 1 for
  the Jacobi matrix T = -D^{-1}(L+U) (checked), so each sweep adds at most
  one rounding difference of each side and the components differ by at
  most 2 k 1e-13 max_m ||scale(x_m)||_inf (the converged-solution check,
  next to the 2-norm check at 1e-12).
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2112_02377_gb300 import jacobi as J
from paper_2112_02377_gb300 import workloads as W

pytestmark = pytest.mark.gpu

RTOL = 1e-13


def _scale(A, b, x):
    S = A.scipy()
    d = S.diagonal()
    off = abs(S) @ np.abs(x) - np.abs(d) * np.abs(x)
    return (np.abs(b) + off) / np.abs(d)


def _t_inf_norm(A):
    S = A.scipy()
    d = np.abs(S.diagonal())
    return float(np.max((abs(S) @ np.ones(A.n) - d) / d))


def _assert_multi_sweep_close(A, b, x_in, x_gpu, x_ref, what):
    """One sweep of every right-hand side (n x nrhs arrays) from the same input."""
    for q in range(b.shape[1]):
        sc = _scale(A, b[:, q], x_in[:, q])
        err = np.abs(x_gpu[:, q] - x_ref[:, q])
        bad = err > RTOL * sc + 1e-300
        assert not bad.any(), (what, q, int(bad.sum()), float(np.max(err / (sc + 1e-300))))


def _per_sweep_check(ctx, mats, rhs, nrhs, sweeps, x0=None):
    """Run `sweeps` single sweeps of the batched context, each compared element
    by element with the oracle's sweep of the GPU's own previous iterate."""
    offs = np.cumsum([0] + [A.n for A in mats])
    if x0 is None:
        x = np.zeros(offs[-1] * nrhs)
    else:
        J.jac_set_x(ctx, x0)
        x = J.jac_get_x(ctx)      # the iterate as stored (y = D x rounds once)
    for k in range(sweeps):
        J.jac_sweep(ctx, 1)
        xg = J.jac_get_x(ctx)
        for s, (A, b) in enumerate(zip(mats, rhs)):
            xin = x[offs[s] * nrhs:offs[s + 1] * nrhs].reshape(A.n, nrhs)
            xout = xg[offs[s] * nrhs:offs[s + 1] * nrhs].reshape(A.n, nrhs)
            y = O.sweep_multi(A, b, xin)[0]
            _assert_multi_sweep_close(A, b, xin, xout, y, (k, s))
        x = xg
    return x


def _batch(nsys, nrhs, seed, lo=4, hi=12):
    rng = np.random.default_rng(seed)
    ms = rng.integers(lo, hi + 1, size=nsys)
    mats, rhs = [], []
    for s, m in enumerate(ms):
        A = W.laplace7(int(m)) if s % 3 else W.diffusion7(int(m), seed=s)
        mats.append(A)
        rhs.append(rng.uniform(-1, 1, size=(A.n, nrhs)))
    return mats, rhs


@pytest.mark.parametrize("nrhs,rows", [(1, 0), (2, 0), (4, 0), (1, 96), (4, 96)])
def test_batched_fp64_each_system_equals_its_own_solve(nrhs, rows):
    mats, rhs = _batch(23, nrhs, seed=nrhs)
    tol = 1e-8
    ctx = J.jac_setup_batched(mats, rhs, J.opts(nrhs=nrhs, sweeps_per_graph=16, tile_rows=rows))
    try:
        k, rel, st = J.jac_solve(ctx, tol, 20000)
        assert st == J.JAC_OK
        x = J.jac_get_x(ctx)
        sweeps, rels = J.jac_get_batch_results(ctx, len(mats) * nrhs)
    finally:
        J.jac_free(ctx)
    off = 0
    for s, (A, b) in enumerate(zip(mats, rhs)):
        assert _t_inf_norm(A) <= 1.0 + 1e-15
        Mo = O.prepare(A)
        xs = x[off * nrhs:(off + A.n) * nrhs].reshape(A.n, nrhs)
        for q in range(nrhs):
            xo, ko, relo, sto = O.solve(A, b[:, q], tol=tol, maxit=20000)
            assert sweeps[s * nrhs + q] == ko, (s, q)
            assert abs(rels[s * nrhs + q] - relo) <= 1e-12
            assert np.linalg.norm(xs[:, q] - xo) <= 1e-12 * np.linalg.norm(xo)
            # element by element: the accumulated rounding bound over ko sweeps
            y, maxsc = np.zeros(A.n), 0.0
            for _ in range(ko):
                maxsc = max(maxsc, float(_scale(A, b[:, q], y).max()))
                y = O.sweep(Mo, b[:, q], y)[0]
            assert np.array_equal(y, xo)
            assert np.all(np.abs(xs[:, q] - xo) <= 2 * ko * RTOL * maxsc), (s, q)
        off += A.n


def test_batched_fixed_sweeps_equal_oracle_sweeps():
    """17 sweeps of 9 systems x 4 right-hand sides, every sweep compared
    element by element with the oracle's sweep of the same input; then 17
    more in one call, bit for bit against a second context run sweep by
    sweep (the graph's sweep count does not change the iterate)."""
    mats, rhs = _batch(9, 4, seed=11)
    x0 = np.random.default_rng(4).uniform(-1, 1, sum(A.n for A in mats) * 4)
    ctx = J.jac_setup_batched(mats, rhs, J.opts(nrhs=4, sweeps_per_graph=5))
    ctx2 = J.jac_setup_batched(mats, rhs, J.opts(nrhs=4, sweeps_per_graph=5))
    try:
        _per_sweep_check(ctx, mats, rhs, 4, 17, x0)
        J.jac_set_x(ctx2, x0)
        for _ in range(17):
            J.jac_sweep(ctx2, 1)
        J.jac_sweep(ctx, 17)
        J.jac_sweep(ctx2, 17)
        assert np.array_equal(J.jac_get_x(ctx), J.jac_get_x(ctx2))
    finally:
        J.jac_free(ctx)
        J.jac_free(ctx2)


def test_batched_mixed_precision_reaches_tolerance():
    mats, rhs = _batch(17, 4, seed=5, lo=6, hi=14)
    tol = 1e-10
    ctx = J.jac_setup_batched(mats, rhs, J.opts(nrhs=4, precision=J.JAC_MIXED, inner_sweeps=32))
    try:
        k, rel, st = J.jac_solve(ctx, tol, 40000)
        assert st == J.JAC_OK
        x = J.jac_get_x(ctx)
        sweeps, rels = J.jac_get_batch_results(ctx, len(mats) * 4)
    finally:
        J.jac_free(ctx)
    off = 0
    for s, (A, b) in enumerate(zip(mats, rhs)):
        xs = x[off * 4:(off + A.n) * 4].reshape(A.n, 4)
        for q in range(4):
            r = b[:, q] - O.spmv(A, xs[:, q])
            assert np.linalg.norm(r) / np.linalg.norm(b[:, q]) <= tol
            assert sweeps[s * 4 + q] % 32 == 0
            ko = O.solve(A, b[:, q], tol=tol, maxit=40000)[1]
            assert ko - 32 <= sweeps[s * 4 + q] <= ko + 2 * 32
        off += A.n


def test_batched_maxit_reports_notconv():
    mats, rhs = _batch(5, 2, seed=2, lo=10, hi=12)
    ctx = J.jac_setup_batched(mats, rhs, J.opts(nrhs=2))
    try:
        k, rel, st = J.jac_solve(ctx, 1e-12, 30)
        assert st == J.JAC_ENOTCONV
        sweeps, rels = J.jac_get_batch_results(ctx, 10)
        assert np.all(sweeps == 30)
    finally:
        J.jac_free(ctx)


def test_batched_autotune_picks_a_geometry_and_stays_exact():
    mats, rhs = _batch(31, 4, seed=3, lo=8, hi=20)
    ctx = J.jac_setup_batched(mats, rhs, J.opts(nrhs=4, autotune=1, sweeps_per_graph=7))
    try:
        st = J.jac_stats(ctx)
        assert st["tile_rows"] in (96, 224) and st["ctas_per_sm"] >= 1
        assert st["sweeps_total"] == 0
        _per_sweep_check(ctx, mats, rhs, 4, 13)
    finally:
        J.jac_free(ctx)


def test_full_size_256_systems_4_rhs_per_sweep_parity():
    """The batched benchmark's workload (256 systems, 6.35 M rows, 4 right-hand
    sides), autotuned: the first sweep from zero, then two sweeps from a
    random iterate, every system and right-hand side against the oracle
    element by element."""
    mats, rhs = W.laplace7_batch(256, seed=0, nrhs=4)
    ctx = J.jac_setup_batched(mats, rhs, J.opts(nrhs=4, autotune=1, sweeps_per_graph=64))
    try:
        _per_sweep_check(ctx, mats, rhs, 4, 1)
        x0 = np.random.default_rng(9).uniform(-1, 1, int(J.jac_stats(ctx)["n"]) * 4)
        _per_sweep_check(ctx, mats, rhs, 4, 2, x0)
    finally:
        J.jac_free(ctx)
