"""Batched solves: many independent systems x several right-hand sides in one
persistent launch.  Every (system, right-hand side) must behave exactly like
its own single-system Jacobi run (Sec. 3 iteration, Algorithm 1 test): same
stopping sweep, same iterate (to the per-sweep tolerance accumulated), same
test value."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2112_02377_gb300 import jacobi as J
from paper_2112_02377_gb300 import workloads as W

pytestmark = pytest.mark.gpu


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
        xs = x[off * nrhs:(off + A.n) * nrhs].reshape(A.n, nrhs)
        for q in range(nrhs):
            xo, ko, relo, sto = O.solve(A, b[:, q], tol=tol, maxit=20000)
            assert sweeps[s * nrhs + q] == ko, (s, q)
            assert abs(rels[s * nrhs + q] - relo) <= 1e-12
            assert np.linalg.norm(xs[:, q] - xo) <= 1e-12 * np.linalg.norm(xo)
        off += A.n


def test_batched_fixed_sweeps_equal_oracle_sweeps():
    mats, rhs = _batch(9, 4, seed=11)
    ctx = J.jac_setup_batched(mats, rhs, J.opts(nrhs=4, sweeps_per_graph=5))
    try:
        J.jac_sweep(ctx, 17)
        x = J.jac_get_x(ctx)
    finally:
        J.jac_free(ctx)
    off = 0
    for A, b in zip(mats, rhs):
        y = np.zeros((A.n, 4))
        for _ in range(17):
            y = O.sweep_multi(A, b, y)[0]
        xs = x[off * 4:(off + A.n) * 4].reshape(A.n, 4)
        assert np.linalg.norm(xs - y) <= 1e-13 * np.linalg.norm(y)
        off += A.n


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
        J.jac_sweep(ctx, 13)
        x = J.jac_get_x(ctx)
    finally:
        J.jac_free(ctx)
    off = 0
    for A, b in zip(mats, rhs):
        y = np.zeros((A.n, 4))
        for _ in range(13):
            y = O.sweep_multi(A, b, y)[0]
        xs = x[off * 4:(off + A.n) * 4].reshape(A.n, 4)
        assert np.linalg.norm(xs - y) <= 1e-13 * np.linalg.norm(y)
        off += A.n


def test_full_size_256_systems_4_rhs_per_sweep_parity():
    """The batched benchmark's workload (256 systems, 6.35 M rows, 4 right-hand
    sides), autotuned: two sweeps of every system and right-hand side against
    the oracle."""
    mats, rhs = W.laplace7_batch(256, seed=0, nrhs=4)
    ctx = J.jac_setup_batched(mats, rhs, J.opts(nrhs=4, autotune=1, sweeps_per_graph=64))
    try:
        J.jac_sweep(ctx, 2)
        x = J.jac_get_x(ctx)
    finally:
        J.jac_free(ctx)
    off = 0
    for A, b in zip(mats, rhs):
        y = np.zeros((A.n, 4))
        for _ in range(2):
            y = O.sweep_multi(A, b, y)[0]
        xs = x[off * 4:(off + A.n) * 4].reshape(A.n, 4)
        assert np.linalg.norm(xs - y) <= 1e-13 * np.linalg.norm(y)
        off += A.n
