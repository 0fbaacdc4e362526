"""GPU parity: the CUDA path against the CPU oracle, through the C ABI.

Tolerances (FP64 path).  One sweep computes x'_i = c_i + sum T_ij x_j with
T_ij = -a_ij / a_ii, c_i = b_i / a_ii and fused multiply-adds; the oracle
computes (1/a_ii)(b_i - sum a_ij x_j) with separately rounded operations.  Both
are backward stable, so for the same input x the two results differ by at most
a few units of roundoff times the row's magnitude
    scale_i = (|b_i| + sum_{j != i} |a_ij x_j|) / |a_ii|,
and we require |x_gpu - x_oracle|_i <= 1e-13 * scale_i (about 450 ulps of the
row scale).  Residual norms: |relres_gpu - relres_oracle| <= 1e-13 *
(||b|| + || |A| |x| ||) / ||b||.  Iterates of different splittings, tilings
and kernel variants are compared bit for bit.
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
    absA = abs(S)
    off = absA @ np.abs(x) - np.abs(d) * np.abs(x)
    return (np.abs(b) + off) / np.abs(d)


def _assert_sweep_close(A, b, x_in, x_gpu, x_ref):
    sc = _scale(A, b, x_in)
    err = np.abs(x_gpu - x_ref)
    bad = err > RTOL * sc + 1e-300
    assert not bad.any(), f"{bad.sum()} rows outside 1e-13*scale; worst ratio {np.max(err / (sc + 1e-300)):.3e}"


def _relres_tol(A, b, x):
    bn = np.linalg.norm(b)
    return RTOL * (bn + np.linalg.norm(abs(A.scipy()) @ np.abs(x))) / (bn if bn > 0 else 1.0)


def _setup(A, b, split, nparts=4, variant=0, sub=(2, 2, 2), **kw):
    s = J.SPLITTINGS[split]
    o = J.opts(variant=variant, **kw)
    node = None
    if s == J.JAC_SUBSTRUCT:
        o.grid[:] = list(A.grid)
        o.subdomains[:] = list(sub)
        node = A.node
    return J.jac_setup(A, b, s, nparts, o, node_of_row=node)


SPLITS = [("bandrow", 4), ("bandrow_nnz", 5), ("substruct", 0)]


def _cases():
    A = W.laplace7(16)
    yield "lap7_16", A, W.solution_and_rhs(A, 0)[1]
    A = W.fe27_deleted(11, seed=2)
    yield "fe27_11", A, W.solution_and_rhs(A, 5)[1]
    A = W.diffusion7((13, 9, 10), seed=4)
    yield "diff7_ragged", A, W.solution_and_rhs(A, 6)[1]
    A = W.convection7(9, peclet=0.9)
    yield "conv7", A, W.solution_and_rhs(A, 8)[1]


@pytest.mark.parametrize("name,A,b", list(_cases()))
@pytest.mark.parametrize("variant", [1, 2, 3])
def test_per_sweep_parity_and_splitting_invariance(name, A, b, variant):
    rng = np.random.default_rng(1)
    x0 = rng.uniform(-1, 1, A.n)
    Mo = O.prepare(A)
    finals = []
    for split, P in SPLITS:
        ctx = _setup(A, b, split, P, variant=variant)
        try:
            J.jac_set_x(ctx, x0)
            x = x0.copy()
            for k in range(6):
                rel = J.jac_sweep(ctx, 1)
                xg = J.jac_get_x(ctx)
                y, ss, mx = O.sweep(Mo, b, x)
                _assert_sweep_close(A, b, x, xg, y)
                assert abs(rel - np.sqrt(ss) / np.linalg.norm(b)) <= _relres_tol(A, b, x)
                x = xg
            J.jac_sweep(ctx, 40)
            finals.append(J.jac_get_x(ctx))
            st = J.jac_stats(ctx)
            assert st["k"] == 46
        finally:
            J.jac_free(ctx)
    for f in finals[1:]:
        assert np.array_equal(f, finals[0])


@pytest.mark.parametrize("name,A,b", list(_cases())[:2])
@pytest.mark.parametrize("lanes", [2, 4, 8])
def test_lanes_per_row_parity_and_splitting_invariance(name, A, b, lanes):
    """Rows summed by 2, 4 or 8 lanes: per-sweep parity with the oracle, and
    the same bits under every splitting and tile balance for a given count."""
    rng = np.random.default_rng(3)
    x0 = rng.uniform(-1, 1, A.n)
    Mo = O.prepare(A)
    finals = []
    for split, P in SPLITS:
        for cps in (2, 3):
            ctx = _setup(A, b, split, P, variant=2, lanes_per_row=lanes, ctas_per_sm=cps, sweeps_per_graph=7)
            try:
                assert J.jac_stats(ctx)["lanes_per_row"] == lanes
                J.jac_set_x(ctx, x0)
                x = x0.copy()
                for k in range(3):
                    rel = J.jac_sweep(ctx, 1)
                    xg = J.jac_get_x(ctx)
                    y, ss, mx = O.sweep(Mo, b, x)
                    _assert_sweep_close(A, b, x, xg, y)
                    assert abs(rel - np.sqrt(ss) / np.linalg.norm(b)) <= _relres_tol(A, b, x)
                    x = xg
                J.jac_sweep(ctx, 30)
                finals.append(J.jac_get_x(ctx))
            finally:
                J.jac_free(ctx)
    for f in finals[1:]:
        assert np.array_equal(f, finals[0])


def test_lanes_per_row_auto_choice_and_mixed():
    A = W.fe27_deleted(14, seed=3)
    xs, b = W.solution_and_rhs(A, 1)
    avg = (A.nnz - A.n) / A.n                    # off-diagonal entries per row
    want = 1
    while want < 8 and avg / (2 * want) >= 8:    # halve the entries per lane while >= 8 remain
        want *= 2
    assert want == 2
    ctx = _setup(A, b, "bandrow_nnz", 4, variant=2)
    try:
        assert J.jac_stats(ctx)["lanes_per_row"] == want
    finally:
        J.jac_free(ctx)
    ctx = _setup(A, b, "bandrow_nnz", 4, variant=2, precision=J.JAC_MIXED, inner_sweeps=32, lanes_per_row=4)
    try:
        k, rel, st = J.jac_solve(ctx, 1e-10, 20000)
        assert st == J.JAC_OK
        x = J.jac_get_x(ctx)
        assert np.linalg.norm(b - O.spmv(A, x)) / np.linalg.norm(b) <= 1e-10
    finally:
        J.jac_free(ctx)
    with pytest.raises(J.JacobiError):
        _setup(A, b, "bandrow", 4, variant=2, tile_rows=480, lanes_per_row=2)


@pytest.mark.parametrize("name,A,b", list(_cases())[:2])
def test_variants_and_graph_batching_are_bit_identical(name, A, b):
    """Every kernel form and every number of sweeps per launch gives the same
    iterate bit for bit.  This also pins the persistent kernel's L1 gathers:
    a launch of many sweeps reads, through L1, rows other CTAs wrote in the
    sweep before, and must equal one launch per sweep and the row kernel
    (a stale L1 line of an older sweep would change the iterate)."""
    outs = []
    for variant, K, rows, cps in [(1, 64, 256, 0), (2, 64, 256, 0), (2, 7, 256, 0), (2, 1, 256, 0),
                                  (2, 64, 256, 3), (2, 64, 480, 0), (2, 5, 480, 0), (2, 64, 224, 0),
                                  (3, 64, 256, 0), (3, 3, 256, 0), (3, 1, 256, 0), (0, 9, 0, 0)]:
        # one lane per row everywhere: the arithmetic the row and halo kernels share
        kw = dict(autotune=1) if variant == 0 else dict(variant=variant, tile_rows=rows, ctas_per_sm=cps)
        ctx = _setup(A, b, "bandrow", 3, sweeps_per_graph=K, lanes_per_row=1, **kw)
        try:
            J.jac_sweep(ctx, 23)
            J.jac_sweep(ctx, 14)
            outs.append(J.jac_get_x(ctx))
        finally:
            J.jac_free(ctx)
    ctx = _setup(A, b, "bandrow", 3, variant=2, lanes_per_row=1)
    try:
        for _ in range(37):
            J.jac_sweep(ctx, 1)
        outs.append(J.jac_get_x(ctx))
    finally:
        J.jac_free(ctx)
    for o in outs[1:]:
        assert np.array_equal(o, outs[0])


@pytest.mark.parametrize("variant", [1, 2, 3])
@pytest.mark.parametrize("split,P", SPLITS)
def test_config1_solve_16cubed_to_1e6(variant, split, P):
    """16^3 7-point Laplace, b = A x* (seed 0), x0 = 0, relative residual 1e-6:
    the oracle (and the DST closed form) take 637 sweeps."""
    A = W.laplace7(16)
    xs, b = W.solution_and_rhs(A, 0)
    xo, ko, relo, sto, hist_o = O.solve(A, b, tol=1e-6, maxit=5000, history=True)
    assert ko == 637
    ctx = _setup(A, b, split, P, variant=variant, history=4096)
    try:
        k, rel, st = J.jac_solve(ctx, 1e-6, 5000)
        assert st == J.JAC_OK and k == ko
        assert abs(rel - relo) <= 1e-12
        xg = J.jac_get_x(ctx)
        assert np.linalg.norm(xg - xo) / np.linalg.norm(xo) < 1e-12
        h = J.jac_get_history(ctx)
        assert len(h) == k + 1
        assert np.max(np.abs(h - hist_o)) < 1e-12
    finally:
        J.jac_free(ctx)


@pytest.mark.parametrize("variant", [1, 2, 3])
def test_paper_q1_count_with_inf_norm(variant):
    """The paper's cube-35937 run: 746 iterations to ||r||_inf < 1e-8 (Sec. 5.2)."""
    A, b = W.q1_laplace(33)
    ctx = _setup(A, b, "bandrow_nnz", 8, variant=variant, norm=J.JAC_NORM_INF)
    try:
        k, rel, st = J.jac_solve(ctx, 1e-8, 10000)
        assert st == J.JAC_OK and k + 1 == 746
    finally:
        J.jac_free(ctx)


@pytest.fixture(scope="module")
def q1_problems():
    return {N: W.q1_laplace(N) for N in (33, 65)}


@pytest.mark.parametrize("N,count", [(33, 746), (65, 2216)])
@pytest.mark.parametrize("P", [8, 64])
@pytest.mark.parametrize("form", ["JB", "JBO", "JSS", "JSS_split"])
def test_paper_replay_counts_every_splitting(q1_problems, N, count, P, form):
    """The paper's Set-1 runs (Sec. 5.2 tables: cube-35937 and cube-274625,
    band-row JB, band-row with dependency lists JBO and substructuring JSS at
    8 and 64 partitions): the Q1 restatement takes 746 and 2216 iterations to
    ||r||_inf < 1e-8 (pinned against the printed counts on the CPU).  With the
    global test every form must reproduce those counts (the paper's JSS
    columns differ because of its local stopping test); the host recomputes
    the residual of the returned iterate."""
    A, b = q1_problems[N]
    sub = (2, 2, 2) if P == 8 else (4, 4, 4)
    o = dict(norm=J.JAC_NORM_INF, sweeps_per_graph=64)
    if form == "JB":
        ctx = _setup(A, b, "bandrow", P, **o)
    elif form == "JBO":
        ctx = _setup(A, b, "bandrow_nnz", P, **o)
    elif form == "JSS":
        ctx = _setup(A, b, "substruct", 0, sub=sub, **o)
    else:
        ctx = J.jac_setup_local(A.n, W.cell_box_locals("q1", N, sub), b, J.opts(**o))
    try:
        st_ = J.jac_stats(ctx)
        assert st_["nparts"] == (P + 1 if form.startswith("JSS") else P)
        k, rel, st = J.jac_solve(ctx, 1e-8, 20000)
        assert st == J.JAC_OK and k + 1 == count
        x = J.jac_get_x(ctx)
    finally:
        J.jac_free(ctx)
    r = np.max(np.abs(b - A.scipy() @ x))
    assert r < 1e-8 and abs(r - rel) <= 1e-3 * rel


def test_maxit_returns_notconv_with_valid_iterate():
    A = W.laplace7(12)
    xs, b = W.solution_and_rhs(A, 2)
    xo, ko, relo, sto = O.solve(A, b, tol=1e-12, maxit=50)
    assert sto == O.JO_ENOTCONV and ko == 50
    ctx = _setup(A, b, "bandrow", 2)
    try:
        k, rel, st = J.jac_solve(ctx, 1e-12, 50)
        assert st == J.JAC_ENOTCONV and k == 50
        assert abs(rel - relo) < 1e-12
        assert np.linalg.norm(J.jac_get_x(ctx) - xo) <= 1e-12 * np.linalg.norm(xo)
    finally:
        J.jac_free(ctx)


# ------------------------------------------------------------ edge cases --

def test_one_by_one_and_diagonal_systems():
    A = W.dense_to_csr(np.array([[4.0]]))
    ctx = _setup(A, np.array([2.0]), "bandrow", 1)
    try:
        k, rel, st = J.jac_solve(ctx, 0.0, 5)
        assert st == J.JAC_OK and k == 1 and rel == 0.0
        assert J.jac_get_x(ctx)[0] == 0.5
    finally:
        J.jac_free(ctx)
    d = np.random.default_rng(3).uniform(1, 2, 700)
    A = W.dense_to_csr(np.diag(d))
    b = np.random.default_rng(4).uniform(-1, 1, 700)
    for variant in (1, 2, 3):
        ctx = _setup(A, b, "bandrow", 7, variant=variant)
        try:
            k, rel, st = J.jac_solve(ctx, 0.0, 5)
            assert st == J.JAC_OK and k == 1
            np.testing.assert_allclose(J.jac_get_x(ctx), O.sweep(A, b, np.zeros(700))[0], rtol=2.3e-16, atol=0)
        finally:
            J.jac_free(ctx)


def test_one_row_per_partition_and_zero_rhs():
    A = W.random_dominant(50, seed=9, density=0.2)
    b = np.random.default_rng(0).uniform(-1, 1, 50)
    x_ref = O.solve(A, b, tol=1e-13, maxit=5000)[0]
    ctx = _setup(A, b, "bandrow", 50)
    try:
        k, rel, st = J.jac_solve(ctx, 1e-13, 5000)
        assert st == J.JAC_OK
        assert np.linalg.norm(J.jac_get_x(ctx) - x_ref) < 1e-12
    finally:
        J.jac_free(ctx)
    ctx = _setup(A, None, "bandrow", 3)
    try:
        k, rel, st = J.jac_solve(ctx, 1e-10, 100)
        assert st == J.JAC_OK and k == 0 and rel == 0.0
    finally:
        J.jac_free(ctx)


def test_device_memory_and_one_based_inputs():
    import torch
    A = W.fe27_deleted(8, seed=7)
    xs, b = W.solution_and_rhs(A, 1)
    ref = None
    for mode in ("host0", "host1", "dev0"):
        if mode == "host0":
            ctx = J.jac_setup(A, b, J.JAC_BANDROW, 3, J.opts())
        elif mode == "host1":
            ctx = J.jac_setup((A.rowptr + 1, A.col + 1, A.val), b, J.JAC_BANDROW, 3, J.opts(), index_base=1)
        else:
            dv = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
            ctx = J.jac_setup((dv(A.rowptr), dv(A.col), dv(A.val)), dv(b), J.JAC_BANDROW, 3, J.opts())
        try:
            J.jac_sweep(ctx, 30)
            if mode == "dev0":
                out = torch.empty(A.n, dtype=torch.float64, device="cuda")
                J.jac_get_x(ctx, out)
                x = out.cpu().numpy()
            else:
                x = J.jac_get_x(ctx)
        finally:
            J.jac_free(ctx)
        if ref is None:
            ref = x
        assert np.array_equal(x, ref)


def test_set_x_resume_equals_continuous_run():
    A = W.laplace7(10)
    xs, b = W.solution_and_rhs(A, 3)
    ctx = _setup(A, b, "substruct", 0)
    try:
        J.jac_sweep(ctx, 30)
        mid = J.jac_get_x(ctx)
        J.jac_sweep(ctx, 20)
        full = J.jac_get_x(ctx)
        J.jac_set_x(ctx, mid)
        J.jac_sweep(ctx, 20)
        # the iterate is held as y = D x: the read-back/write-back round trip
        # rounds once each way, which the contraction does not amplify
        res = J.jac_get_x(ctx)
        assert np.max(np.abs(res - full)) <= 4e-16 * np.max(np.abs(full)) * 20
        assert J.jac_stats(ctx)["k"] == 20
    finally:
        J.jac_free(ctx)


def test_errors_singular_duplicate_diagonal_divergence():
    M = np.array([[1.0, 2.0], [3.0, 0.0]])
    with pytest.raises(J.JacobiError) as ei:
        J.jac_setup(W.dense_to_csr(M), np.ones(2), J.JAC_BANDROW, 1)
    assert ei.value.status == J.JAC_ESINGULAR
    A = W.dense_to_csr(np.array([[2.0, 1.0], [1.0, 2.0]]))
    B = W.CSR(2, np.array([0, 3, 5], np.int32), np.array([0, 0, 1, 0, 1], np.int32),
              np.array([1.0, 1.0, 1.0, 1.0, 2.0]))
    with pytest.raises(J.JacobiError) as ei:
        J.jac_setup(B, np.ones(2), J.JAC_BANDROW, 1)
    assert ei.value.status == J.JAC_EINVAL
    # rho(T) >> 1: the iterate overflows and the residual becomes Inf/NaN
    D = np.array([[1e-200, 1.0, 0.0], [1.0, 1e-200, 1.0], [0.0, 1.0, 1e-200]])
    for variant in (1, 2, 3):
        ctx = J.jac_setup(W.dense_to_csr(D), np.ones(3), J.JAC_BANDROW, 1, J.opts(variant=variant))
        try:
            with pytest.raises(J.JacobiError) as ei:
                J.jac_solve(ctx, 1e-8, 100)
            assert ei.value.status == J.JAC_ENUMERIC
        finally:
            J.jac_free(ctx)


def test_grid_barrier_timeout_is_reported_and_recoverable():
    """One CTA never arrives at the grid barrier (host-set hook); the others
    give up after a short bounded wait and the call reports JAC_ETIMEOUT."""
    A = W.laplace7(24)
    xs, b = W.solution_and_rhs(A, 0)
    for variant in (2, 3):
        ctx = J.jac_setup(A, b, J.JAC_BANDROW, 4, J.opts(variant=variant, fault_skip_cta=1, timeout_cycles=20_000_000))
        try:
            with pytest.raises(J.JacobiError) as ei:
                J.jac_sweep(ctx, 5)
            assert ei.value.status == J.JAC_ETIMEOUT
        finally:
            J.jac_free(ctx)
    ctx = _setup(A, b, "bandrow", 4, variant=2)
    try:
        J.jac_sweep(ctx, 5)
        x = J.jac_get_x(ctx)
        y = np.zeros(A.n)
        for _ in range(5):
            y = O.sweep(A, b, y)[0]
        assert np.linalg.norm(x - y) <= 1e-13 * np.linalg.norm(y)
    finally:
        J.jac_free(ctx)


# ------------------------------------------------ neighbour-synchronised sweeps ----

NS = dict(variant=2, sync=J.JAC_SYNC_NEIGHBOUR)


@pytest.mark.parametrize("name,A,b", list(_cases()))
@pytest.mark.parametrize("split,P", SPLITS)
def test_neighbour_sync_sweeps_equal_grid_barrier_sweeps(name, A, b, split, P):
    """Neighbour flags order the sweeps exactly like the grid barrier: the same
    iterate bits after any number of sweeps and graph launch sizes, and the
    same residual of the last pre-update iterate."""
    rng = np.random.default_rng(4)
    x0 = rng.uniform(-1, 1, A.n)
    ref = _setup(A, b, split, P, variant=2, sweeps_per_graph=64)
    try:
        J.jac_set_x(ref, x0)
        rel_ref = J.jac_sweep(ref, 29)
        x_ref = J.jac_get_x(ref)
    finally:
        J.jac_free(ref)
    for K, cps in [(64, 2), (1, 3), (2, 2), (7, 3)]:
        ctx = _setup(A, b, split, P, sweeps_per_graph=K, ctas_per_sm=cps, **NS)
        try:
            assert J.jac_stats(ctx)["sync"] == J.JAC_SYNC_NEIGHBOUR
            J.jac_set_x(ctx, x0)
            rel = J.jac_sweep(ctx, 29)
            assert np.array_equal(J.jac_get_x(ctx), x_ref), (K, cps)
            assert rel == rel_ref
            assert J.jac_stats(ctx)["k"] == 29
        finally:
            J.jac_free(ctx)


@pytest.mark.parametrize("split,P", SPLITS)
@pytest.mark.parametrize("K", [1, 3, 64, 256])
def test_neighbour_sync_solve_stops_where_the_grid_barrier_stops(split, P, K):
    """The test of x^k is taken a sweep late but x^k is kept: same stopping
    sweep, same iterate, same residual history as the grid barrier (and the
    oracle's 637 sweeps to 1e-6 at 16^3)."""
    A = W.laplace7(16)
    xs, b = W.solution_and_rhs(A, 0)
    out = []
    for kw in (dict(variant=2), NS):
        ctx = _setup(A, b, split, P, sweeps_per_graph=K, history=1000, **kw)
        try:
            k, rel, st = J.jac_solve(ctx, 1e-6, 5000)
            out.append((k, rel, st, J.jac_get_x(ctx), J.jac_get_history(ctx)))
        finally:
            J.jac_free(ctx)
    (k0, r0, s0, x0, h0), (k1, r1, s1, x1, h1) = out
    assert s0 == s1 == J.JAC_OK and k0 == k1 == 637
    assert r0 == r1 and np.array_equal(x0, x1) and np.array_equal(h0, h1)


def test_neighbour_sync_maxit_and_resume():
    A = W.fe27_deleted(11, seed=2)
    xs, b = W.solution_and_rhs(A, 5)
    res = []
    for kw in (dict(variant=2), NS):
        ctx = _setup(A, b, "bandrow_nnz", 5, sweeps_per_graph=5, **kw)
        try:
            k, rel, st = J.jac_solve(ctx, 1e-30, 23)
            assert st == J.JAC_ENOTCONV and k == 23
            k2, rel2, st2 = J.jac_solve(ctx, 1e-30, 31)      # continues from x^23
            res.append((k, rel, k2, rel2, J.jac_get_x(ctx)))
        finally:
            J.jac_free(ctx)
    assert res[0][:4] == res[1][:4] and np.array_equal(res[0][4], res[1][4])


def test_neighbour_sync_timeout_is_reported_and_recoverable():
    A = W.laplace7(12)
    xs, b = W.solution_and_rhs(A, 0)
    ctx = _setup(A, b, "bandrow", 4, fault_skip_cta=3, timeout_cycles=20_000_000, **NS)
    try:
        with pytest.raises(J.JacobiError) as e:
            J.jac_sweep(ctx, 10)
        assert e.value.status == J.JAC_ETIMEOUT
    finally:
        J.jac_free(ctx)
    ctx = _setup(A, b, "bandrow", 4, **NS)
    try:
        J.jac_sweep(ctx, 10)
        y = np.zeros(A.n)
        for _ in range(10):
            y = O.sweep(A, b, y)[0]
        assert np.linalg.norm(J.jac_get_x(ctx) - y) <= 1e-13 * np.linalg.norm(y)
    finally:
        J.jac_free(ctx)


# ------------------------------------------------ asynchronous relaxation ----
# Not deterministic: checked by converged-solution parity, never by iterates.

@pytest.mark.parametrize("name,A,b", list(_cases()))
@pytest.mark.parametrize("split,P", SPLITS)
def test_async_relaxation_converges_to_the_oracle_solution(name, A, b, split, P):
    tol = 1e-10
    xo, ko, relo, sto = O.solve(A, b, tol=tol, maxit=200000)
    ctx = _setup(A, b, split, P, variant=2, sync=J.JAC_SYNC_ASYNC, sweeps_per_graph=16)
    try:
        assert J.jac_stats(ctx)["sync"] == J.JAC_SYNC_ASYNC
        k, rel, st = J.jac_solve(ctx, tol, 200000)
        assert st == J.JAC_OK and 0 < k <= 4 * ko
        x = J.jac_get_x(ctx)
        true_rel = np.linalg.norm(b - O.spmv(A, x)) / np.linalg.norm(b)
        assert true_rel <= tol * (1 + 1e-6)                  # the certified test value is exact
        assert abs(rel - true_rel) <= 1e-13 * (1 + np.linalg.norm(np.abs(A.scipy()) @ np.abs(x)) / np.linalg.norm(b))
        # both are tol-accurate solutions of A x = b
        assert np.linalg.norm(x - xo) <= 1e-6 * np.linalg.norm(xo)
    finally:
        J.jac_free(ctx)


def test_async_relaxation_maxit_and_fixed_passes():
    A = W.laplace7(14)
    xs, b = W.solution_and_rhs(A, 2)
    ctx = _setup(A, b, "bandrow", 4, variant=2, sync=J.JAC_SYNC_ASYNC, sweeps_per_graph=8)
    try:
        k, rel, st = J.jac_solve(ctx, 1e-30, 40)
        assert st == J.JAC_ENOTCONV and k == 40
        x = J.jac_get_x(ctx)
        true_rel = np.linalg.norm(b - O.spmv(A, x)) / np.linalg.norm(b)
        assert abs(rel - true_rel) <= 1e-12 and true_rel < 1.0
        J.jac_set_x(ctx, None)
        J.jac_sweep(ctx, 25)
        assert J.jac_stats(ctx)["k"] == 25
        x = J.jac_get_x(ctx)
        assert np.all(np.isfinite(x))
        assert np.linalg.norm(b - O.spmv(A, x)) < np.linalg.norm(b)
    finally:
        J.jac_free(ctx)


@pytest.mark.parametrize("stages", [2, 3, 4])
def test_every_stage_count_with_every_sync_mode(stages):
    """Each (stages, sync) pair runs its own kernel instantiation: neighbour
    sync gives the grid barrier's bits, asynchronous relaxation converges."""
    A = W.fe27_deleted(12, seed=4)
    xs, b = W.solution_and_rhs(A, 3)
    out = {}
    for sync in (J.JAC_SYNC_GRID, J.JAC_SYNC_NEIGHBOUR):
        ctx = _setup(A, b, "bandrow_nnz", 4, variant=2, stages=stages, sync=sync, sweeps_per_graph=9)
        try:
            assert J.jac_stats(ctx)["stages"] == stages
            J.jac_sweep(ctx, 31)
            out[sync] = J.jac_get_x(ctx)
        finally:
            J.jac_free(ctx)
    assert np.array_equal(out[J.JAC_SYNC_GRID], out[J.JAC_SYNC_NEIGHBOUR])
    ctx = _setup(A, b, "bandrow_nnz", 4, variant=2, stages=stages, sync=J.JAC_SYNC_ASYNC, sweeps_per_graph=9)
    try:
        k, rel, st = J.jac_solve(ctx, 1e-10, 100000)
        assert st == J.JAC_OK
        x = J.jac_get_x(ctx)
        assert np.linalg.norm(b - O.spmv(A, x)) / np.linalg.norm(b) <= 1e-10 * (1 + 1e-6)
    finally:
        J.jac_free(ctx)


@pytest.mark.parametrize("kw", [dict(variant=1), dict(variant=2), dict(variant=3), dict(variant=2, lanes_per_row=4),
                                dict(variant=2, stages=2, lanes_per_row=2), dict(variant=2, sync=J.JAC_SYNC_NEIGHBOUR),
                                dict(variant=2, sync=J.JAC_SYNC_ASYNC), dict(variant=2, precision=J.JAC_MIXED),
                                dict(variant=2, tile_rows=480, precision=J.JAC_MIXED)])
def test_no_kernel_writes_past_a_device_vector(kw):
    """Canary bytes after every device vector (opts.debug) survive sweeps and
    solves of every kernel form, on a ragged problem."""
    A = W.fe27_deleted(10, seed=6)
    xs, b = W.solution_and_rhs(A, 4)
    ctx = _setup(A, b, "bandrow_nnz", 3, debug=1, sweeps_per_graph=5, inner_sweeps=8, **kw)
    try:
        J.jac_sweep(ctx, 13)
        J.jac_solve(ctx, 1e-9, 20000)
        J.jac_set_x(ctx, xs)
        J.jac_sweep(ctx, 2)
        assert np.all(np.isfinite(J.jac_get_x(ctx)))
    finally:
        J.jac_free(ctx)


def test_nan_in_b_is_reported():
    A = W.laplace7(8)
    xs, b = W.solution_and_rhs(A, 0)
    b[17] = np.nan
    ctx = _setup(A, b, "bandrow", 2, variant=2)
    try:
        with pytest.raises(J.JacobiError) as e:
            J.jac_solve(ctx, 1e-8, 1000)
        assert e.value.status == J.JAC_ENUMERIC
    finally:
        J.jac_free(ctx)


# ------------------------------------------------ irregular matrices, option mix ----

_OPTION_MIX = [dict(variant=1), dict(variant=3), dict(variant=2), dict(variant=2, ctas_per_sm=3),
               dict(variant=2, tile_rows=224), dict(variant=2, tile_rows=480),
               dict(variant=2, sync=J.JAC_SYNC_NEIGHBOUR), dict(variant=2, stages=2, sync=J.JAC_SYNC_NEIGHBOUR),
               dict(variant=2, lanes_per_row=2), dict(variant=2, lanes_per_row=2, stages=3),
               dict(variant=2, lanes_per_row=4, ctas_per_sm=3), dict(variant=2, lanes_per_row=8, stages=2)]


@pytest.mark.parametrize("seed", [1, 2])
def test_irregular_rows_under_every_option_mix(seed):
    """Row lengths from 2 to 200 plus rows longer than a staged tile, entries
    in random order: per-sweep parity with the oracle for every kernel form,
    and one bit pattern per lane count across kernel forms and splittings."""
    A = W.random_irregular(20000 if seed == 1 else 7000, seed)
    rng = np.random.default_rng(seed + 40)
    b = rng.uniform(-1, 1, A.n)
    x0 = rng.uniform(-1, 1, A.n)
    Mo = O.prepare(A)
    y1 = O.sweep(Mo, b, x0)[0]
    y2, ss2, _ = O.sweep(Mo, b, y1)
    finals = {}
    for i, kw in enumerate(_OPTION_MIX):
        split, P = [("bandrow", 5), ("bandrow_nnz", 13)][i % 2]
        ctx = _setup(A, b, split, P, sweeps_per_graph=3, **kw)
        try:
            J.jac_set_x(ctx, x0)
            J.jac_sweep(ctx, 1)
            x1 = J.jac_get_x(ctx)
            _assert_sweep_close(A, b, x0, x1, y1)
            J.jac_set_x(ctx, y1)                    # the oracle's iterate as input: a clean second step
            rel = J.jac_sweep(ctx, 1)
            _assert_sweep_close(A, b, y1, J.jac_get_x(ctx), y2)
            assert abs(rel - np.sqrt(ss2) / np.linalg.norm(b)) <= _relres_tol(A, b, y1)
            J.jac_set_x(ctx, x0)
            J.jac_sweep(ctx, 11)
            finals.setdefault(J.jac_stats(ctx)["lanes_per_row"], []).append((kw, split, J.jac_get_x(ctx)))
        finally:
            J.jac_free(ctx)
    for group in finals.values():
        kw0, s0, f0 = group[0]
        for kw, sp, f in group[1:]:
            bad = np.flatnonzero(f != f0)
            assert bad.size == 0, (f"{kw} {sp} differs from {kw0} {s0} in {bad.size} rows, first {bad[:5]}, "
                                   f"row lengths {np.diff(A.rowptr)[bad[:5]]}")


def test_autotune_reports_its_choice_and_starts_from_zero():
    A = W.laplace7(24)
    xs, b = W.solution_and_rhs(A, 1)
    for prec in (J.JAC_FP64, J.JAC_MIXED):
        ctx = _setup(A, b, "bandrow_nnz", 4, autotune=1, precision=prec, inner_sweeps=16)
        try:
            st = J.jac_stats(ctx)
            assert (st["variant"], st["tile_rows"]) in [(2, 256), (2, 224), (2, 480), (3, 256)]
            assert st["ctas_per_sm"] >= 1 and st["sweeps_total"] == 0
            x = J.jac_get_x(ctx)
            assert not np.any(x)
            if prec == J.JAC_FP64:
                J.jac_sweep(ctx, 6)
                y = np.zeros(A.n)
                for _ in range(6):
                    y = O.sweep(A, b, y)[0]
                assert np.linalg.norm(J.jac_get_x(ctx) - y) <= 1e-13 * np.linalg.norm(y)
            else:
                k, rel, s = J.jac_solve(ctx, 1e-9, 20000)
                assert s == J.JAC_OK and rel <= 1e-9
        finally:
            J.jac_free(ctx)


# ---------------------------------------------------- mixed precision ----

@pytest.mark.parametrize("variant,rows", [(1, 256), (2, 256), (2, 224), (2, 480), (3, 256)])
def test_mixed_precision_reaches_1e10(variant, rows):
    A = W.laplace7(16)
    xs, b = W.solution_and_rhs(A, 0)
    x64, k64, rel64, st64 = O.solve(A, b, tol=1e-10, maxit=20000)
    ctx = _setup(A, b, "bandrow", 4, variant=variant, precision=J.JAC_MIXED, inner_sweeps=64, tile_rows=rows)
    try:
        k, rel, st = J.jac_solve(ctx, 1e-10, 20000)
        assert st == J.JAC_OK
        x = J.jac_get_x(ctx)
        r = b - O.spmv(A, x)
        assert np.linalg.norm(r) / np.linalg.norm(b) <= 1e-10
        assert abs(rel - np.linalg.norm(r) / np.linalg.norm(b)) < 1e-13
        assert k > 0 and k % 64 == 0 and k64 - 64 <= k <= k64 + 3 * 64
        assert np.linalg.norm(x - x64) / np.linalg.norm(x64) < 1e-8
    finally:
        J.jac_free(ctx)


# ------------------------------------------------- full size (160^3) -----

@pytest.fixture(scope="module")
def big():
    A = W.laplace7(160)
    xs, b = W.solution_and_rhs(A, 0)
    return A, b


def test_full_size_160cubed_per_sweep_parity_all_splittings(big):
    """The benchmark's workload and launch configuration (autotuned contexts,
    64 sweeps per graph): every element of three consecutive sweeps against the
    oracle fed the same input, for each splitting; then 61 more sweeps and the
    iterates compared bit for bit (also against the staged-halo kernel and
    neighbour-synchronised sweeps)."""
    A, b = big
    rng = np.random.default_rng(11)
    x0 = rng.uniform(-1, 1, A.n)
    Mo = O.prepare(A)
    finals = {}
    # the autotuned runs are grouped by the lane count they chose; the pinned
    # one-lane runs make sure all three splittings meet in one group
    runs = [(("bandrow", 64), dict(autotune=1)), (("bandrow_nnz", 64), dict(autotune=1)),
            (("substruct", 0), dict(autotune=1)), (("bandrow", 64), dict(variant=3)),
            (("substruct", 0), dict(variant=2, lanes_per_row=1, sync=J.JAC_SYNC_NEIGHBOUR)),
            (("bandrow_nnz", 64), dict(variant=2, lanes_per_row=1))]
    for (split, P), kw in runs:
        ctx = _setup(A, b, split, P, sub=(4, 4, 4), sweeps_per_graph=64, **kw)
        try:
            J.jac_set_x(ctx, x0)
            x = x0
            for k in range(3):
                rel = J.jac_sweep(ctx, 1)
                xg = J.jac_get_x(ctx)
                y, ss, mx = O.sweep(Mo, b, x)
                _assert_sweep_close(A, b, x, xg, y)
                assert abs(rel - np.sqrt(ss) / np.linalg.norm(b)) <= _relres_tol(A, b, x)
                x = xg
            J.jac_sweep(ctx, 61)
            finals.setdefault(J.jac_stats(ctx)["lanes_per_row"], []).append((split, J.jac_get_x(ctx)))
        finally:
            J.jac_free(ctx)
    assert {sp for sp, _ in finals[1]} == {"bandrow", "bandrow_nnz", "substruct"}
    for group in finals.values():
        for sp, f in group[1:]:
            assert np.array_equal(f, group[0][1]), sp


def test_full_size_160cubed_solve_stops_at_the_closed_form_count(big):
    """The benchmark's time-to-1e-8 workload: the DST closed form of the 160^3
    residual history crosses 1e-8 after 42,745 sweeps, with a relative margin
    above 7e-5 on both sides (pinned on the CPU), so the FP64 solve must stop
    at exactly that sweep; its iterate then has relres <= 1e-8 when checked
    on the host, and matches the reported value."""
    A, b = big
    ctx = _setup(A, b, "bandrow_nnz", 64)
    try:
        k, rel, st = J.jac_solve(ctx, 1e-8, 60000)
        assert st == J.JAC_OK and k == 42745
        x = J.jac_get_x(ctx)
    finally:
        J.jac_free(ctx)
    r = b - A.scipy() @ x
    relx = np.linalg.norm(r) / np.linalg.norm(b)
    assert relx <= 1e-8 and abs(relx - rel) <= 1e-6 * rel


def test_full_size_fe27_128cubed_per_sweep_parity():
    """FE-like 27-point operator at 128^3 nodes (2.1 M rows, 53.8 M entries),
    autotuned as in the secondary benchmark: two sweeps element by element."""
    A = W.fe27_deleted(128, seed=0)
    xs, b = W.solution_and_rhs(A, 0)
    rng = np.random.default_rng(12)
    x0 = rng.uniform(-1, 1, A.n)
    Mo = O.prepare(A)
    ctx = _setup(A, b, "bandrow_nnz", 64, autotune=1, sweeps_per_graph=64)
    try:
        J.jac_set_x(ctx, x0)
        x = x0
        for k in range(2):
            rel = J.jac_sweep(ctx, 1)
            xg = J.jac_get_x(ctx)
            y, ss, mx = O.sweep(Mo, b, x)
            _assert_sweep_close(A, b, x, xg, y)
            assert abs(rel - np.sqrt(ss) / np.linalg.norm(b)) <= _relres_tol(A, b, x)
            x = xg
    finally:
        J.jac_free(ctx)


@pytest.mark.parametrize("mode", ["fp64", "mixed", "async"])
def test_full_size_fe27_128cubed_solve_reaches_1e10(mode):
    """The FE-27 benchmark's solves at full size (2.1 M rows, 53.8 M entries)
    in its configuration (autotuned, nnz-balanced bands, graphs of 256 sweeps,
    mixed cycles of 128): each reports relres <= 1e-10, and the residual of the
    returned iterate recomputed on the host agrees with it to 1e-3 relative
    (the host's rounding floor is near 1e-15 here)."""
    A = W.fe27_deleted(128, seed=0)
    xs, b = W.solution_and_rhs(A, 0)
    prec = J.JAC_MIXED if mode == "mixed" else J.JAC_FP64
    sync = J.JAC_SYNC_ASYNC if mode == "async" else J.JAC_SYNC_GRID
    ctx = _setup(A, b, "bandrow_nnz", 64, autotune=1, precision=prec, sync=sync, inner_sweeps=128,
                 sweeps_per_graph=256)
    try:
        k, rel, st = J.jac_solve(ctx, 1e-10, 200000)
        assert st == J.JAC_OK and 0 < rel <= 1e-10
        x = J.jac_get_x(ctx)
    finally:
        J.jac_free(ctx)
    relx = np.linalg.norm(b - A.scipy() @ x) / np.linalg.norm(b)
    assert abs(relx - rel) <= 1e-3 * rel
