"""GPU parity of substructuring with the interface block split between
subdomains (Sec. 4.3: local matrices, two-step product, weighted interface
dot), through jac_setup_local, against the CPU oracle's split sweep and the
assembled sweep.  Tolerances as in test_gpu_parity: 1e-13 of each row's scale
per sweep; iterates of one lane count bit for bit across kernel geometries."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2112_02377_gb300 import jacobi as J
from paper_2112_02377_gb300 import workloads as W
from test_gpu_parity import RTOL, _assert_sweep_close, _relres_tol

pytestmark = pytest.mark.gpu


def _ctx(A, locs, b, **kw):
    return J.jac_setup_local(A.n, locs, b, J.opts(**kw))


_GEOMS = [dict(), dict(ctas_per_sm=3), dict(stages=3), dict(stages=2), dict(lanes_per_row=2),
          dict(lanes_per_row=2, ctas_per_sm=3), dict(lanes_per_row=4), dict(lanes_per_row=4, stages=2)]


@pytest.mark.parametrize("kind,m,sub", [("laplace7", 20, (2, 2, 2)), ("laplace7", (23, 17, 19), (3, 2, 4)),
                                        ("q1", 17, (2, 2, 2)), ("q1", 21, (4, 4, 4))])
def test_split_sweeps_match_the_oracles_and_agree_across_geometries(kind, m, sub):
    if kind == "laplace7":
        A = W.laplace7(m)
        b = W.solution_and_rhs(A, 3)[1]
    else:
        A, b = W.q1_laplace(m)
    locs = W.cell_box_locals(kind, m, sub)
    P = O.split_prepare(locs, A.n)
    rng = np.random.default_rng(7)
    x0 = rng.uniform(-1, 1, A.n)
    y1, ss1, mx1 = O.split_sweep(P, b, x0)
    y2, ss2, mx2 = O.split_sweep(P, b, y1)
    a1 = O.sweep(A, b, x0)[0]
    finals = {}
    for kw in _GEOMS:
        ctx = _ctx(A, locs, b, sweeps_per_graph=3, **kw)
        try:
            st = J.jac_stats(ctx)
            assert st["interface_rows"] == P.interface().size
            assert st["halo_entries"] == int(P.mult[P.mult >= 2].sum())
            assert st["nparts"] == len(locs) + 1 and st["splitting"] == J.JAC_SUBSTRUCT
            J.jac_set_x(ctx, x0)
            J.jac_sweep(ctx, 1)
            g1 = J.jac_get_x(ctx)
            _assert_sweep_close(A, b, x0, g1, y1)         # the oracle's split sweep
            _assert_sweep_close(A, b, x0, g1, a1)         # the assembled sweep
            J.jac_set_x(ctx, y1)
            rel = J.jac_sweep(ctx, 1)
            _assert_sweep_close(A, b, y1, J.jac_get_x(ctx), y2)
            assert abs(rel - np.sqrt(ss2) / np.linalg.norm(b)) <= _relres_tol(A, b, y1)
            J.jac_set_x(ctx, x0)
            J.jac_sweep(ctx, 9)
            finals.setdefault(st["lanes_per_row"], []).append((kw, J.jac_get_x(ctx)))
        finally:
            J.jac_free(ctx)
    assert set(finals) == {1, 2, 4}
    for group in finals.values():
        kw0, f0 = group[0]
        for kw, f in group[1:]:
            assert np.array_equal(f, f0), f"{kw} differs from {kw0}"
    # across lane counts: rounding only
    ref = finals[1][0][1]
    for L in (2, 4):
        assert np.max(np.abs(finals[L][0][1] - ref)) <= 1e-12 * np.max(np.abs(ref))


@pytest.mark.parametrize("lanes", [1, 2, 4])
def test_one_subdomain_is_the_unsplit_sweep_bit_for_bit(lanes):
    A = W.laplace7(18)
    b = W.solution_and_rhs(A, 4)[1]
    locs = W.cell_box_locals("laplace7", 18, (1, 1, 1))
    ctx = _ctx(A, locs, b, lanes_per_row=lanes)
    ref = J.jac_setup(A, b, J.JAC_BANDROW, 1, J.opts(variant=2, lanes_per_row=lanes))
    try:
        for c in (ctx, ref):
            J.jac_sweep(c, 13)
        assert J.jac_stats(ctx)["interface_rows"] == 0
        assert np.array_equal(J.jac_get_x(ctx), J.jac_get_x(ref))
        assert J.jac_stats(ctx)["last_relres"] == J.jac_stats(ref)["last_relres"]
    finally:
        J.jac_free(ctx)
        J.jac_free(ref)


def test_corner_rows_of_eight_subdomains_fill_a_warp_with_four_lanes():
    A = W.laplace7(9)
    b = W.solution_and_rhs(A, 2)[1]
    locs = W.cell_box_locals("laplace7", 9, (2, 2, 2))
    P = O.split_prepare(locs, A.n)
    assert P.mult.max() == 8
    x0 = np.random.default_rng(1).uniform(-1, 1, A.n)
    ctx = _ctx(A, locs, b, lanes_per_row=4)
    try:
        J.jac_set_x(ctx, x0)
        J.jac_sweep(ctx, 1)
        _assert_sweep_close(A, b, x0, J.jac_get_x(ctx), O.split_sweep(P, b, x0)[0])
    finally:
        J.jac_free(ctx)


def test_split_solve_and_set_b():
    m, sub = 24, (4, 4, 4)
    A = W.laplace7(m)
    xs, b = W.solution_and_rhs(A, 5)
    locs = W.cell_box_locals("laplace7", m, sub)
    ctx = _ctx(A, locs, b, debug=1)
    try:
        k, rel, st = J.jac_solve(ctx, 1e-8, 20000)
        _, k0, rel0, _ = O.solve(A, b, None, tol=1e-8, maxit=20000)
        assert st == J.JAC_OK and abs(k - k0) <= 1 and rel <= 1e-8
        assert np.max(np.abs(J.jac_get_x(ctx) - xs)) <= 1e-6
        # a new right-hand side, same iterate
        b2 = np.random.default_rng(2).uniform(-1, 1, A.n)
        x = J.jac_get_x(ctx)
        J.jac_set_b(ctx, b2)
        J.jac_set_x(ctx, x)
        J.jac_sweep(ctx, 1)
        P = O.split_prepare(locs, A.n)
        _assert_sweep_close(A, b2, x, J.jac_get_x(ctx), O.split_sweep(P, b2, x)[0])
        # the adjoint gradient needs the caller's assembled pattern, which a
        # context built from local matrices does not hold
        with pytest.raises(J.JacobiError) as ei:
            J.jac_adjoint_grad(ctx, np.zeros(A.n), np.zeros(A.n), np.zeros(A.nnz))
        assert ei.value.status == J.JAC_EINVAL and "local matrices" in str(ei.value)
    finally:
        J.jac_free(ctx)


@pytest.mark.parametrize("sub", [(2, 2, 2), (4, 4, 4)])
def test_q1_replay_count_on_the_gpu(sub):
    """33^3-node Set-1 problem, ||r||_inf < 1e-8 (Sec. 5.2 tables: 746)."""
    A, b = W.q1_laplace(33)
    locs = W.cell_box_locals("q1", 33, sub)
    ctx = _ctx(A, locs, b, norm=J.JAC_NORM_INF, autotune=1)
    try:
        k, rel, st = J.jac_solve(ctx, 1e-8, 5000)
        assert st == J.JAC_OK and abs((k + 1) - 746) <= 1
        P = O.split_prepare(locs, A.n)
        x_o, k_o, rel_o, _ = O.split_solve(P, b, None, tol=1e-8, maxit=5000, norm=0)
        assert abs(k - k_o) <= 1
        assert np.max(np.abs(J.jac_get_x(ctx) - x_o)) <= 1e-10 * np.max(np.abs(x_o))
    finally:
        J.jac_free(ctx)


def test_full_size_160_cube_split_sweep_against_oracle_and_substructuring():
    """The 160^3 7-point system split into 4x4x4 cell boxes (the bench's
    substructuring configuration): one autotuned sweep against the whole
    oracle split sweep, and against the node-based substructuring kernel."""
    m, sub = 160, (4, 4, 4)
    A = W.laplace7(m)
    b = W.solution_and_rhs(A, 0)[1]
    locs = W.cell_box_locals("laplace7", m, sub)
    x0 = np.random.default_rng(11).uniform(-1, 1, A.n)
    P = O.split_prepare(locs, A.n)
    y1, ss1, _ = O.split_sweep(P, b, x0)
    ctx = _ctx(A, locs, b, autotune=1)
    o = J.opts(variant=2, grid=A.grid, subdomains=sub)
    ref = J.jac_setup(A, b, J.JAC_SUBSTRUCT, 0, o)
    try:
        for c in (ctx, ref):
            J.jac_set_x(c, x0)
        rel = J.jac_sweep(ctx, 1)
        J.jac_sweep(ref, 1)
        g = J.jac_get_x(ctx)
        _assert_sweep_close(A, b, x0, g, y1)
        _assert_sweep_close(A, b, x0, g, J.jac_get_x(ref))
        assert abs(rel - np.sqrt(ss1) / np.linalg.norm(b)) <= _relres_tol(A, b, x0)
        st = J.jac_stats(ctx)
        assert st["interface_rows"] == P.interface().size == 226107
    finally:
        J.jac_free(ctx)
        J.jac_free(ref)


def _random_unstructured_locals(n, nsub, seed):
    """Overlapping random node sets (rows held by 1 to 5 subdomains), random
    local patterns stored in random order, off-diagonal pieces of both signs,
    local diagonals sharing a dominance margin; plus an empty subdomain and
    one made only of rows that other subdomains also hold."""
    rng = np.random.default_rng(seed)
    owner = rng.integers(0, nsub, n)
    sets = [list(np.flatnonzero(owner == s)) for s in range(nsub)]
    for g in rng.choice(n, n // 5, replace=False):         # extra holders
        for s in rng.choice(nsub, rng.integers(1, 5), replace=False):
            if g not in sets[s]:
                sets[s].append(g)
    shared = [g for g in range(n) if sum(g in S for S in sets) >= 2][:40]
    sets.append(shared)                                    # only interface rows
    sets.append([])                                        # empty
    locs = []
    for S in sets:
        nodes = np.array(sorted(S), dtype=np.int32)
        nl = nodes.size
        rowptr, col, val = [0], [], []
        for l in range(nl):
            k = int(rng.integers(0, min(nl, 30))) if nl > 1 else 0
            others = rng.choice([j for j in range(nl) if j != l], k, replace=False) if k else []
            ent = [(int(j), float(rng.uniform(-1, 1))) for j in others] + [(l, 0.0)]
            rng.shuffle(ent)
            for j, v in ent:
                col.append(j)
                val.append(v)
            rowptr.append(len(col))
        locs.append(W.LocalCSR(nl, np.array(rowptr, np.int32), np.array(col, np.int32), np.array(val), nodes))
    absoff = np.zeros(n)
    for L in locs:
        rows = np.repeat(np.arange(L.n), np.diff(L.rowptr))
        np.add.at(absoff, L.l2g[rows], np.where(L.col != rows, np.abs(L.val), 0.0))
    for L in locs:
        rows = np.repeat(np.arange(L.n), np.diff(L.rowptr))
        dg = L.col == rows
        L.val[dg] = (1.2 * absoff[L.l2g[rows[dg]]] + 0.5) * rng.uniform(0.3, 1.0, dg.sum())
    return locs


@pytest.mark.parametrize("lanes", [1, 2, 4])
def test_unstructured_local_matrices_with_mixed_sign_pieces(lanes):
    n = 6000
    locs = _random_unstructured_locals(n, 9, 5)
    P = O.split_prepare(locs, n)
    assert P.mult.max() >= 4 and locs[-1].n == 0
    rng = np.random.default_rng(3)
    b, x0 = rng.uniform(-1, 1, n), rng.uniform(-1, 1, n)
    y1, ss1, _ = O.split_sweep(P, b, x0)
    # scale of a row: |b| + sum over subdomains of |local off-diagonal terms|, over |d|
    sc = np.abs(b).copy()
    for L in locs:
        rows = np.repeat(np.arange(L.n), np.diff(L.rowptr))
        off = L.col != rows
        np.add.at(sc, L.l2g[rows[off]], np.abs(L.val[off] * x0[L.l2g[L.col[off]]]))
    sc /= np.abs(P.d)
    ctx = J.jac_setup_local(n, locs, b, J.opts(lanes_per_row=lanes, debug=1))
    try:
        J.jac_set_x(ctx, x0)
        rel = J.jac_sweep(ctx, 1)
        err = np.abs(J.jac_get_x(ctx) - y1)
        assert np.all(err <= RTOL * sc), f"worst {np.max(err / sc):.3e}"
        assert abs(rel - np.sqrt(ss1) / np.linalg.norm(b)) <= 1e-12 * np.sqrt(ss1) / np.linalg.norm(b) + 1e-15
        k, r, st = J.jac_solve(ctx, 1e-10, 5000)
        xs, ko, ro, _ = O.split_solve(P, b, None, tol=1e-10, maxit=5000)
        assert st == J.JAC_OK and abs(k - ko) <= 1
        assert np.max(np.abs(J.jac_get_x(ctx) - xs)) <= 1e-9 * np.max(np.abs(xs))
    finally:
        J.jac_free(ctx)


def _star(nsub, seed):
    """nsub subdomains, each holding row 0 and one row of its own; row 0
    is then a group of nsub slot rows."""
    rng = np.random.default_rng(seed)
    locs = []
    for s in range(nsub):
        a = rng.uniform(0.1, 1.0)
        locs.append(W.LocalCSR(2, np.array([0, 2, 4], np.int32), np.array([1, 0, 0, 1], np.int32),
                               np.array([-a, 3.0, -a, 2.0 + a]), np.array([0, s + 1], np.int32)))
    return locs, nsub + 1


def _everything_shared(n, seed):
    """Two subdomains that both hold every row, each with half of a
    diagonally dominant tridiagonal matrix: no interior rows at all."""
    rng = np.random.default_rng(seed)
    locs = []
    for s in range(2):
        rowptr, col, val = [0], [], []
        for i in range(n):
            for j in (i - 1, i, i + 1):
                if 0 <= j < n:
                    col.append(j)
                    val.append(2.5 + rng.uniform(0, 0.5) if j == i else -0.5 * rng.uniform(0.5, 1.0))
            rowptr.append(len(col))
        locs.append(W.LocalCSR(n, np.array(rowptr, np.int32), np.array(col, np.int32), np.array(val),
                               np.arange(n, dtype=np.int32)))
    return locs, n


@pytest.mark.parametrize("case", ["one_row", "star32", "star8_lanes4", "everything_shared"])
def test_split_degenerate_layouts(case):
    if case == "one_row":
        locs = [W.LocalCSR(1, np.array([0, 1], np.int32), np.array([0], np.int32), np.array([4.0]),
                           np.array([0], np.int32))]
        n, lanes = 1, 1
    elif case == "star32":
        locs, n = _star(32, 1)
        lanes = 1
    elif case == "star8_lanes4":
        locs, n = _star(8, 2)
        lanes = 4
    else:
        locs, n = _everything_shared(700, 3)
        lanes = 1
    P = O.split_prepare(locs, n)
    rng = np.random.default_rng(9)
    b, x0 = rng.uniform(-1, 1, n), rng.uniform(-1, 1, n)
    ctx = J.jac_setup_local(n, locs, b, J.opts(lanes_per_row=lanes, debug=1))
    try:
        st = J.jac_stats(ctx)
        assert st["interface_rows"] == int((P.mult >= 2).sum())
        x = x0.copy()
        J.jac_set_x(ctx, x0)
        for _ in range(3):
            y_ref, ss, _ = O.split_sweep(P, b, x)
            rel = J.jac_sweep(ctx, 1)
            g = J.jac_get_x(ctx)
            sc = np.abs(b) + 1.0
            for L in locs:
                rows = np.repeat(np.arange(L.n), np.diff(L.rowptr))
                off = L.col != rows
                np.add.at(sc, L.l2g[rows[off]], np.abs(L.val[off] * x[L.l2g[L.col[off]]]))
            assert np.all(np.abs(g - y_ref) <= RTOL * sc / np.abs(P.d))
            assert abs(rel - np.sqrt(ss) / np.linalg.norm(b)) <= 1e-12 * (np.sqrt(ss) / np.linalg.norm(b)) + 1e-15
            x = y_ref
    finally:
        J.jac_free(ctx)
