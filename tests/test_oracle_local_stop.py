"""Pins of the oracle's local-convergence stopping rule (Sec. 3, the parallel
form of Algorithm 1) and of the row sets each partition holds.

Each partition p tests max_{i in R_p} |r_i| <= tol on the rows R_p it holds.
Rule "all" (every partition passes at once) must equal the global
infinity-norm test whenever the sets cover every row; rule "first" stops at
the first sweep in which some partition passes, which is the smallest of the
sweeps at which each partition alone would stop.  Box row sets (the nodes of
a subdomain's box of cells) are checked against the separator-plane rule."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2112_02377_gb300 import workloads as W


def _cuts(g, p):
    return [(t * g) // p for t in range(1, p)]


@pytest.mark.parametrize("grid,sub", [((7, 9, 11), (2, 3, 2)), ((8, 8, 8), (4, 4, 4)), ((5, 6, 7), (1, 2, 3)),
                                      ((31, 31, 31), (2, 2, 2))])
def test_box_row_sets_follow_the_separator_planes(grid, sub):
    """A node lies in 2 boxes per cut plane through it and in one box per axis
    otherwise; along an axis its boxes are those whose closed node range
    [c_t, c_{t+1}] holds it.  Interior nodes sit in their own subdomain's box
    only; the sets cover every node."""
    gx, gy, gz = grid
    n = gx * gy * gz
    sets = O.box_row_sets(grid, sub, n)
    mult = np.zeros(n, dtype=np.int64)
    for S in sets:
        mult[S] += 1
    node = np.arange(n)
    X, Y, Z = node % gx, (node // gx) % gy, node // (gx * gy)
    expect = np.ones(n, dtype=np.int64)
    for c, g, p in ((X, gx, sub[0]), (Y, gy, sub[1]), (Z, gz, sub[2])):
        expect *= np.where(np.isin(c, _cuts(g, p)), 2, 1)
    assert np.array_equal(mult, expect)

    def boxes(c, g, p):
        lo = [0] + _cuts(g, p)
        hi = _cuts(g, p) + [g - 1]
        return {t for t in range(p) if lo[t] <= c <= hi[t]}

    rng = np.random.default_rng(0)
    for i in rng.choice(n, 200, replace=False):
        want = {bx + sub[0] * (by + sub[1] * bz) for bx in boxes(X[i], gx, sub[0]) for by in boxes(Y[i], gy, sub[1])
                for bz in boxes(Z[i], gz, sub[2])}
        got = {s for s, S in enumerate(sets) if i in set(S.tolist())}
        assert got == want
    perm, part_ptr = O.substructure(grid, sub, n)
    for s in range(len(sets)):
        inner = perm[part_ptr[s]:part_ptr[s + 1]]
        assert set(inner.tolist()) <= set(sets[s].tolist())
        assert np.all(mult[inner] == 1)


def _problem():
    A = W.laplace7((9, 8, 7))
    xs, b = W.solution_and_rhs(A, 3)
    return A, b


def test_one_partition_is_the_global_test():
    A, b = _problem()
    xg, kg, rg, sg = O.solve(A, b, tol=1e-8, maxit=5000, norm=0)
    x, k, p, loc, st = O.solve_local(A, b, [np.arange(A.n)], tol=1e-8, maxit=5000)
    assert st == O.JO_OK and (k, p) == (kg, 0) and loc == rg
    assert np.array_equal(x, xg)


@pytest.mark.parametrize("kind", ["bands", "boxes"])
def test_all_partitions_at_once_is_the_global_test(kind):
    A, b = _problem()
    sets = (O.band_row_sets(O.band_row_parts(A.n, 7)) if kind == "bands"
            else O.box_row_sets(A.grid, (2, 2, 3), A.n))
    xg, kg, rg, sg = O.solve(A, b, tol=1e-8, maxit=5000, norm=0)
    x, k, p, loc, st = O.solve_local(A, b, sets, tol=1e-8, maxit=5000, rule="all")
    assert st == O.JO_OK and k == kg and loc == rg
    assert np.array_equal(x, xg)


@pytest.mark.parametrize("kind", ["bands", "boxes"])
def test_first_partition_is_the_earliest_single_partition_stop(kind):
    """Rule "first" stops at min over p of the sweep at which partition p
    alone passes, never after the global test, and names a partition that
    passes there (the one with the smallest local value)."""
    A, b = _problem()
    sets = (O.band_row_sets(O.band_row_parts(A.n, 5)) if kind == "bands"
            else O.box_row_sets(A.grid, (3, 2, 2), A.n))
    x, k, p, loc, st = O.solve_local(A, b, sets, tol=1e-8, maxit=5000)
    alone = [O.solve_local(A, b, [S], tol=1e-8, maxit=5000)[1] for S in sets]
    kg = O.solve(A, b, tol=1e-8, maxit=5000, norm=0)[1]
    assert st == O.JO_OK and k == min(alone) <= kg
    assert alone[p] == min(alone) and loc <= 1e-8


def test_local_stop_against_dense_brute_force():
    """A random diagonally dominant 14 x 14 system and overlapping row sets,
    iterated densely with numpy (x' = x + D^{-1}(b - A x)): the same stopping
    sweep and partition under both rules (the local values at the stopping
    sweeps are well away from tol, so rounding cannot move them)."""
    rng = np.random.default_rng(5)
    n = 14
    M = rng.uniform(-1, 1, (n, n)) * (rng.uniform(size=(n, n)) < 0.4)
    np.fill_diagonal(M, 0.0)
    np.fill_diagonal(M, np.abs(M).sum(axis=1) * 1.3 + 0.1)
    A = W.dense_to_csr(M)
    b = rng.uniform(-1, 1, n)
    sets = [np.array([0, 1, 2, 3, 4]), np.array([4, 5, 6, 7, 8, 9]), np.array([9, 10, 11, 12, 13, 0])]
    tol = 1e-6
    d = np.diag(M)
    for rule in ("first", "all"):
        x = np.zeros(n)
        for kk in range(2000):
            r = b - M @ x
            loc = np.array([np.max(np.abs(r[S])) for S in sets])
            pick = int(np.argmin(loc)) if rule == "first" else int(np.argmax(loc))
            if loc[pick] <= tol:
                break
            x = x + r / d
        assert abs(loc[pick] - tol) > 1e-3 * tol
        xo, k, p, lo, st = O.solve_local(A, b, sets, tol=tol, maxit=2000, rule=rule)
        assert st == O.JO_OK and (k, p) == (kk, pick)
        assert np.allclose(xo, x, rtol=0, atol=1e-12)


def test_rows_held_by_no_partition_are_rejected():
    A, b = _problem()
    with pytest.raises(ValueError):
        O.solve_local(A, b, [np.arange(5), np.array([], dtype=np.int64)])
