"""Stopping on local convergence (JAC_STOP_LOCAL) against the oracle.

Reading (Sec. 3, the parallel form of Algorithm 1, and the substructuring
counts of the Sec. 5.2 tables): every partition tests max |r_i| <= tol on the
rows it holds -- its band, or the nodes of its box of grid cells under
substructuring -- and the solve ends at the first sweep in which one
partition passes.  The GPU must stop at the oracle's sweep, name the same
partition, report its local value, and return the oracle's iterate.

Tolerances: the GPU's iterate after k sweeps is compared element by element
with the oracle's within 2 k 1e-13 max_m ||scale(x_m)||_inf (||T||_inf <= 1
for these operators: each sweep adds at most one rounding difference of each
side; scale_i = (|b_i| + sum_{j != i} |a_ij x_j|) / |a_ii|); local values
within 1e-13 of the largest row magnitude |b_i| + sum_j |a_ij x_j| plus what
that iterate difference can move them.  The stopping sweeps are checked to
lie well away from a rounding tie (the oracle's local value at the sweep
before the stop exceeds tol by more than the bound)."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2112_02377_gb300 import jacobi as J
from paper_2112_02377_gb300 import workloads as W

pytestmark = pytest.mark.gpu

RTOL = 1e-13


@pytest.fixture(scope="module")
def q1_33():
    return W.q1_laplace(33)


def _scale(A, b, x):
    S = A.scipy()
    d = S.diagonal()
    off = abs(S) @ np.abs(x) - np.abs(d) * np.abs(x)
    return (np.abs(b) + off) / np.abs(d)


def _oracle_run(A, b, sets, tol, maxit=20000):
    """The oracle's local-stop solve, plus the largest row scale over its
    iterates and the local value one sweep before the stop (tie margin)."""
    x, k, p, loc, st = O.solve_local(A, b, sets, tol=tol, maxit=maxit)
    Mo = O.prepare(A)
    y, maxsc, before = np.zeros(A.n), 0.0, np.inf
    absA = abs(A.scipy())
    rowmag = 0.0
    for m in range(k + 1):
        maxsc = max(maxsc, float(_scale(A, b, y).max()))
        rowmag = max(rowmag, float(np.max(np.abs(b) + absA @ np.abs(y))))
        yn, ss, mx, r = O.sweep(Mo, b, y, want_r=True)
        if m == k - 1:
            before = min(float(np.max(np.abs(r[S]))) for S in sets)
        if m < k:
            y = yn
    assert np.array_equal(y, x)
    return x, k, p, loc, st, maxsc, before, rowmag


def _setup(A, b, form, P, sub, **kw):
    o = dict(norm=J.JAC_NORM_INF, stop=J.JAC_STOP_LOCAL, sweeps_per_graph=64)
    o.update(kw)
    if form == "JB":
        return J.jac_setup(A, b, J.JAC_BANDROW, P, J.opts(**o))
    if form == "JBO":
        return J.jac_setup(A, b, J.JAC_BANDROW_NNZ, P, J.opts(**o))
    return J.jac_setup(A, b, J.JAC_SUBSTRUCT, 0, J.opts(grid=A.grid, subdomains=sub, **o))


def _sets(A, form, P, sub):
    if form == "JB":
        return O.band_row_sets(O.band_row_parts(A.n, P))
    if form == "JBO":
        return O.band_row_sets(O.band_nnz_parts(A.rowptr, P))
    return O.box_row_sets(A.grid, sub, A.n)


@pytest.mark.parametrize("form,P,sub", [("JB", 8, None), ("JB", 64, None), ("JBO", 8, None), ("JBO", 64, None),
                                        ("JSS", 8, (2, 2, 2)), ("JSS", 16, (4, 2, 2)), ("JSS", 32, (4, 4, 2)),
                                        ("JSS", 64, (4, 4, 4))])
def test_paper_replay_local_stop_matches_the_oracle(q1_33, form, P, sub):
    """The Q1 33^3-node replay (||r||_inf < 1e-8) under every splitting."""
    A, b = q1_33
    tol = 1e-8
    sets = _sets(A, form, P, sub)
    xo, ko, po, loco, sto, maxsc, before, rowmag = _oracle_run(A, b, sets, tol)
    assert sto == O.JO_OK
    bound = 2 * ko * RTOL * maxsc
    vtol = RTOL * rowmag + float(np.max(abs(A.scipy()) @ np.full(A.n, bound)))
    assert before > tol + vtol and loco < tol - vtol    # no rounding tie at the stopping sweep
    ctx = _setup(A, b, form, P, sub)
    try:
        k, rel, st = J.jac_solve(ctx, tol, 20000)
        stt = J.jac_stats(ctx)
        x = J.jac_get_x(ctx)
    finally:
        J.jac_free(ctx)
    assert st == J.JAC_OK and k == ko
    assert stt["stop"] == J.JAC_STOP_LOCAL and stt["stop_part"] == po
    assert abs(stt["stop_local"] - loco) <= vtol
    assert np.all(np.abs(x - xo) <= bound)
    # the reported test value is still the global one, of the same iterate
    assert abs(rel - np.max(np.abs(b - A.scipy() @ x))) <= vtol


@pytest.mark.parametrize("form,P,sub", [("JSS", 64, (4, 4, 4)), ("JBO", 8, None)])
def test_paper_replay_65cubed_local_stop_matches_the_oracle(form, P, sub):
    """The Q1 65^3-node replay (the paper's cube-274625 table, ||r||_inf <
    1e-8) with the local test: stopping sweep and partition as the oracle's."""
    A, b = W.q1_laplace(65)
    sets = _sets(A, form, P, sub)
    xo, ko, po, loco, sto = O.solve_local(A, b, sets, tol=1e-8, maxit=20000)
    assert sto == O.JO_OK
    ctx = _setup(A, b, form, P, sub)
    try:
        k, rel, st = J.jac_solve(ctx, 1e-8, 20000)
        stt = J.jac_stats(ctx)
        x = J.jac_get_x(ctx)
    finally:
        J.jac_free(ctx)
    assert st == J.JAC_OK and k == ko and stt["stop_part"] == po
    assert np.linalg.norm(x - xo) <= 1e-10 * np.linalg.norm(xo)


@pytest.mark.parametrize("lanes,cps,stages", [(1, 2, 0), (1, 3, 0), (2, 2, 2), (2, 2, 3), (4, 2, 0)])
def test_local_stop_every_geometry_stops_at_the_same_sweep(q1_33, lanes, cps, stages):
    """Each lane count, CTA count and stage count of the local-stop kernel
    form: same stopping sweep and partition as the oracle (4x4x4 boxes)."""
    A, b = q1_33
    sets = _sets(A, "JSS", 64, (4, 4, 4))
    xo, ko, po, loco, sto = O.solve_local(A, b, sets, tol=1e-8, maxit=20000)
    ctx = _setup(A, b, "JSS", 64, (4, 4, 4), variant=2, lanes_per_row=lanes, ctas_per_sm=cps, stages=stages,
                 sweeps_per_graph=37)
    try:
        st_ = J.jac_stats(ctx)
        assert st_["lanes_per_row"] == lanes
        k, rel, st = J.jac_solve(ctx, 1e-8, 20000)
        assert st == J.JAC_OK and k == ko and J.jac_stats(ctx)["stop_part"] == po
    finally:
        J.jac_free(ctx)


def test_local_stop_autotuned_and_resumed(q1_33):
    """An autotuned context stops at the oracle's sweep; a second solve from
    the returned iterate stops at once (the local test still passes), and
    jac_sweep runs its k sweeps without a test."""
    A, b = q1_33
    sets = _sets(A, "JB", 8, None)
    xo, ko, po, loco, sto = O.solve_local(A, b, sets, tol=1e-8, maxit=20000)
    ctx = _setup(A, b, "JB", 8, None, autotune=1)
    try:
        k, rel, st = J.jac_solve(ctx, 1e-8, 20000)
        assert st == J.JAC_OK and k == ko and J.jac_stats(ctx)["stop_part"] == po
        k2, rel2, st2 = J.jac_solve(ctx, 1e-8, 20000)
        assert st2 == J.JAC_OK and k2 == ko
        J.jac_set_x(ctx, None)
        J.jac_sweep(ctx, 40)
        assert J.jac_stats(ctx)["k"] == 40
    finally:
        J.jac_free(ctx)


def test_local_stop_maxit_and_global_equivalence(q1_33):
    """maxit before any partition passes: JAC_ENOTCONV and no partition named.
    One partition holding every row (a single band) is the global test."""
    A, b = q1_33
    ctx = _setup(A, b, "JB", 8, None)
    try:
        k, rel, st = J.jac_solve(ctx, 1e-8, 100)
        assert st == J.JAC_ENOTCONV and k == 100 and J.jac_stats(ctx)["stop_part"] == -1
    finally:
        J.jac_free(ctx)
    kg = O.solve(A, b, tol=1e-8, maxit=20000, norm=0)[1]
    ctx = _setup(A, b, "JB", 1, None)
    try:
        k, rel, st = J.jac_solve(ctx, 1e-8, 20000)
        assert st == J.JAC_OK and k == kg and J.jac_stats(ctx)["stop_part"] == 0
    finally:
        J.jac_free(ctx)
