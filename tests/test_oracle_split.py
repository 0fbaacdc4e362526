"""Pins of the oracle's split-interface substructuring (Sec. 4.3): local
matrices A_s with A33 = sum_s A33^(s), the two-step product and the weighted
interface dot product.  CPU only."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2112_02377_gb300 import workloads as W


def _dense_from_locals(locs, n):
    """sum_s P_s^T A_s P_s, entry by entry (brute force)."""
    A = np.zeros((n, n))
    for L in locs:
        for l in range(L.n):
            for k in range(L.rowptr[l], L.rowptr[l + 1]):
                A[L.l2g[l], L.l2g[L.col[k]]] += L.val[k]
    return A


def _random_locals(seed):
    """Three subdomains over 14 nodes with overlapping node sets (node 6 in all
    three), random sparse local patterns stored in random order, and local
    diagonals large enough that the assembled matrix is strictly dominant."""
    rng = np.random.default_rng(seed)
    sets = [np.arange(0, 7), np.arange(5, 11), np.array([6, 9, 10, 11, 12, 13])]
    locs = []
    for nodes in sets:
        nl = nodes.size
        rowptr, col, val = [0], [], []
        for l in range(nl):
            others = [j for j in range(nl) if j != l and rng.random() < 0.5]
            ent = [(j, rng.uniform(-1, 1)) for j in others] + [(l, 0.0)]
            rng.shuffle(ent)
            for j, v in ent:
                col.append(j)
                val.append(v)
            rowptr.append(len(col))
        locs.append(W.LocalCSR(nl, np.array(rowptr, np.int32), np.array(col, np.int32), np.array(val),
                               nodes.astype(np.int32)))
    # local diagonals: each subdomain carries a share of the dominance margin
    n = 14
    off = np.abs(_dense_from_locals(locs, n)).sum(axis=1)
    for L in locs:
        for l in range(L.n):
            for k in range(L.rowptr[l], L.rowptr[l + 1]):
                if L.col[k] == l:
                    L.val[k] = (1.5 * off[L.l2g[l]] + 0.1) * rng.uniform(0.2, 1.0)
    return locs, n


@pytest.mark.parametrize("m,sub", [(9, (2, 2, 2)), ((7, 5, 6), (3, 1, 2)), (12, (4, 4, 4)), (6, (1, 1, 1))])
def test_laplace7_local_matrices_reassemble_exactly(m, sub):
    A = W.laplace7(m)
    locs = W.cell_box_locals("laplace7", m, sub)
    assert len(locs) == sub[0] * sub[1] * sub[2]
    assert np.array_equal(_dense_from_locals(locs, A.n), A.scipy().toarray())
    # the shared nodes are the separator planes of the node-based substructuring
    P = O.split_prepare(locs, A.n)
    perm, part_ptr = O.substructure(A.grid, sub, A.n)
    S = sub[0] * sub[1] * sub[2]
    assert np.array_equal(P.interface(), np.sort(perm[part_ptr[S]:part_ptr[S + 1]]))
    assert set(np.unique(P.mult)) <= {1, 2, 4, 8}


@pytest.mark.parametrize("N,sub", [(9, (2, 2, 2)), (12, (3, 3, 3))])
def test_q1_local_matrices_reassemble_the_assembled_stiffness(N, sub):
    A, _ = W.q1_laplace(N)
    locs = W.cell_box_locals("q1", N, sub)
    D = _dense_from_locals(locs, A.n)
    ref = A.scipy().toarray()
    assert np.max(np.abs(D - ref)) <= 4e-16 * np.max(np.abs(ref))
    # every local row sums to zero away from the Dirichlet boundary (a pure
    # Neumann element assembly): check one subdomain's rows with all 27 entries
    L = locs[0]
    full = np.diff(L.rowptr) == 21            # 27 minus the 6 zero edge couplings, all inside the box
    sums = np.add.reduceat(L.val, L.rowptr[:-1])[full]
    assert full.any() and np.max(np.abs(sums)) <= 1e-16 * np.max(np.abs(L.val))


def test_one_subdomain_reduces_to_the_plain_sweep_bit_for_bit():
    A = W.laplace7(10)
    rng = np.random.default_rng(3)
    b, x = rng.uniform(-1, 1, A.n), rng.uniform(-1, 1, A.n)
    P = O.split_prepare(W.cell_box_locals("laplace7", 10, (1, 1, 1)), A.n)
    y, ss, mx = O.split_sweep(P, b, x)
    y0, ss0, mx0 = O.sweep(A, b, x)
    assert np.array_equal(y, y0) and ss == ss0 and mx == mx0


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_split_sweep_matches_dense_jacobi_on_overlapping_random_locals(seed):
    locs, n = _random_locals(seed)
    A = _dense_from_locals(locs, n)
    d = np.diag(A).copy()
    rng = np.random.default_rng(seed + 10)
    b, x = rng.uniform(-1, 1, n), rng.uniform(-1, 1, n)
    P = O.split_prepare(locs, n)
    assert list(np.bincount(P.mult, minlength=4)[1:4]) == [10, 3, 1]   # node 6 in three subdomains
    assert np.allclose(P.d, d, rtol=1e-15, atol=0)
    y, ss, mx, r = O.split_sweep(P, b, x, want_r=True)
    y_ref = (b - (A - np.diag(d)) @ x) / d
    r_ref = b - A @ x
    scale = np.abs(A) @ np.abs(x) + np.abs(b)
    assert np.all(np.abs(y - y_ref) <= 1e-14 * scale / np.abs(d))
    assert np.all(np.abs(r - r_ref) <= 1e-14 * scale)
    # the weighted interface dot counts every node once
    assert abs(ss - np.sum(r_ref ** 2)) <= 1e-13 * np.sum(r_ref ** 2)
    assert abs(mx - np.max(np.abs(r_ref))) <= 1e-14 * np.max(scale)
    # converged solution against dense LU
    xs, k, rel, st = O.split_solve(P, b, None, tol=1e-13, maxit=10000)
    assert st == O.JO_OK
    assert np.allclose(xs, np.linalg.solve(A, b), rtol=0, atol=1e-12)


@pytest.mark.parametrize("sub", [(2, 2, 2), (4, 4, 4)])
def test_q1_replay_count_with_split_interface(sub):
    """The paper's synchronous count for the 33^3-node Set-1 problem with the
    residual test ||D(x^{k+1}-x^k)||_inf < 1e-8 (Sec. 5.2 tables: 746; the
    paper notes every synchronous variant should give the same count for any
    number of processes)."""
    A, b = W.q1_laplace(33)
    P = O.split_prepare(W.cell_box_locals("q1", 33, sub), A.n)
    x, k, rel, st = O.split_solve(P, b, None, tol=1e-8, maxit=5000, norm=0)
    assert st == O.JO_OK and abs((k + 1) - 746) <= 1
    x0, k0, rel0, st0 = O.solve(A, b, None, tol=1e-8, maxit=5000, norm=0)
    assert abs(k - k0) <= 1
    assert np.max(np.abs(x - x0)) <= 1e-10 * np.max(np.abs(x0))


def test_split_prepare_rejects_uncovered_nodes_and_zero_diagonals():
    locs = W.cell_box_locals("laplace7", 4, (2, 1, 1))
    with pytest.raises(ValueError):
        O.split_prepare(locs[:1], 64)
    bad = [W.LocalCSR(L.n, L.rowptr, L.col, np.where(L.col == np.repeat(np.arange(L.n), np.diff(L.rowptr)), 0.0,
                                                       L.val), L.l2g) for L in locs]
    with pytest.raises(ZeroDivisionError):
        O.split_prepare(bad, 64)
