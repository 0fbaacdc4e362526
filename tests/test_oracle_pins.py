"""Pins of the CPU oracle to facts outside itself.

Each test checks the oracle against something the paper or the mathematics
fixes: values printed in the paper (tests/golden), the closed-form spectrum of
the 7-point Laplacian (discrete sine transform), dense LU solutions, the
fixed-point property of the iteration, and brute force on tiny inputs.
"""
import numpy as np
import pytest
import scipy.fft as F
import scipy.sparse as sp

from conftest import golden_path
from oracle import oracle as O
from paper_2112_02377_gb300 import workloads as W


# ---------------------------------------------------------------- fixtures --

def _read_csr_golden():
    out = {"A": []}
    for line in open(golden_path("csr_example_5x5.txt")):
        line = line.split("#")[0].strip()
        if not line:
            continue
        key, *vals = line.split()
        if key == "A":
            out["A"].append([float(v) for v in vals])
        elif key == "n":
            out["n"] = int(vals[0])
        else:
            out[key] = [float(v) for v in vals] if key == "AA" else [int(v) for v in vals]
    return out


def _read_dependency_golden():
    rows, recv, send, bands = {}, {}, {}, None
    for line in open(golden_path("dependency_10x10_3bands.txt")):
        line = line.split("#")[0].strip()
        if not line:
            continue
        if line.startswith("row"):
            head, cols = line.split(":")
            rows[int(head.split()[1])] = [int(c) for c in cols.split()]
        elif line.startswith("bands"):
            bands = [int(v) for v in line.split()[1:]]
        elif line.startswith("recv") or line.startswith("send"):
            head, nodes = line.split(":")
            kind, a, _, b = head.split()
            (recv if kind == "recv" else send)[(int(a), int(b))] = [int(v) for v in nodes.split()]
    return rows, bands, recv, send


def _dst_history(grid, xstar, K):
    """Closed-form relative residual history of Jacobi on the 7-point Laplacian.

    With x0 = 0 and b = A x*, the error e_k = (I - A/6)^k (-x*); in the DST-I
    eigenbasis A has eigenvalues lam = sum_d (2 - 2 cos(pi j_d/(g_d+1))), so
    ||r_k||_2 = ||lam * (1 - lam/6)^k * z||_2 with z = DST(x*).
    """
    gx, gy, gz = grid
    z = F.dstn(xstar.reshape(gz, gy, gx), type=1, norm="ortho")
    ev = [2.0 - 2.0 * np.cos(np.pi * np.arange(1, g + 1) / (g + 1)) for g in (gz, gy, gx)]
    lam = ev[0][:, None, None] + ev[1][None, :, None] + ev[2][None, None, :]
    mu = 1.0 - lam / 6.0
    bn = np.sqrt(np.sum((lam * z) ** 2))
    return np.array([np.sqrt(np.sum((lam * mu ** k * z) ** 2)) / bn for k in range(K)])


# -------------------------------------------------------------------- CSR --

def test_csr_worked_example_matches_printed_arrays():
    g = _read_csr_golden()
    dense = np.array(g["A"])
    # the printed 1-based AA/JA/IA rebuild the printed dense matrix
    rebuilt = np.zeros((g["n"], g["n"]))
    IA, JA, AA = g["IA"], g["JA"], g["AA"]
    assert IA[-1] == len(AA) + 1
    for i in range(g["n"]):
        for k in range(IA[i] - 1, IA[i + 1] - 1):
            rebuilt[i, JA[k] - 1] = AA[k]
    np.testing.assert_array_equal(rebuilt, dense)
    # the input helper produces the same arrays (0-based) from the dense matrix
    A = W.dense_to_csr(W.paper_csr_example())
    np.testing.assert_array_equal(A.rowptr + 1, IA)
    np.testing.assert_array_equal(A.col + 1, JA)
    np.testing.assert_array_equal(A.val, AA)
    # oracle product on this CSR equals the dense product (LAPACK/BLAS route)
    x = np.array([0.5, -1.0, 2.0, 0.25, -3.0])
    np.testing.assert_allclose(O.spmv(A, x), dense @ x, rtol=0, atol=1e-13)


def test_csr_example_sweep_against_dense_split():
    """One sweep on the printed matrix equals the splitting form of Eq. (3.3),
    x' = M^{-1} N x + M^{-1} b with M = D, N = D - A, built densely."""
    dense = W.paper_csr_example()
    A = W.dense_to_csr(dense)
    b = np.array([1.0, 2.0, -1.0, 0.5, 3.0])
    x = np.array([0.1, -0.2, 0.3, -0.4, 0.5])
    M = np.diag(np.diag(dense))
    N = M - dense
    ref = np.linalg.solve(M, N @ x + b)
    y, ss, mx, r = O.sweep(A, b, x, want_r=True)
    np.testing.assert_allclose(y, ref, rtol=1e-15, atol=1e-15)
    np.testing.assert_allclose(r, b - dense @ x, rtol=0, atol=1e-13)
    assert ss == pytest.approx(np.sum((b - dense @ x) ** 2), rel=1e-14)
    assert mx == pytest.approx(np.max(np.abs(b - dense @ x)), rel=1e-15)


# --------------------------------------------------------- dependency lists --

def test_dependency_lists_reproduce_paper_tables():
    rows, bands, recv_g, send_g = _read_dependency_golden()
    pat = W.paper_pattern_10x10()
    for r, cols in rows.items():
        assert sorted(np.nonzero(pat[r - 1])[0] + 1) == cols
    parts = O.band_row_parts(10, 3)
    assert list(parts + 1) == bands           # floor(p n / P) gives the printed 3/3/4 bands
    A = W.dense_to_csr(pat.astype(float) + 10 * np.eye(10))
    recv, send = O.dependency_lists(A.rowptr, A.col, parts)
    got_recv = {(p + 1, q + 1): list(v + 1) for p in range(3) for q, v in recv[p].items()}
    got_send = {(q + 1, p + 1): list(v + 1) for q in range(3) for p, v in send[q].items()}
    assert got_recv == recv_g
    assert got_send == send_g


def test_partitioned_sweep_detects_incomplete_dependency_list():
    A = W.laplace7(6)
    xs, b = W.solution_and_rhs(A, 1)
    parts = O.band_row_parts(A.n, 4)
    recv, _ = O.dependency_lists(A.rowptr, A.col, parts)
    hp, h = O.halo_of(recv)
    rows = np.arange(A.n)
    O.partitioned_sweep(A, b, xs, parts, rows, hp, h)      # complete lists: fine
    h2 = h.copy()
    h2[0] = h2[1]                                          # plant a missing entry
    with pytest.raises(LookupError):
        O.partitioned_sweep(A, b, xs, parts, rows, hp, h2)


# ----------------------------------------------------------- splittings ----

def test_band_row_parts_brute_force():
    for n in range(1, 40):
        for P in range(1, n + 1):
            parts = O.band_row_parts(n, P)
            sizes = np.diff(parts)
            assert parts[0] == 0 and parts[-1] == n
            assert sizes.min() >= n // P and sizes.max() <= -(-n // P)


def test_band_nnz_parts_brute_force():
    rng = np.random.default_rng(5)
    for trial in range(60):
        n = int(rng.integers(1, 30))
        lens = rng.integers(0, 9, size=n)
        rp = np.concatenate([[0], np.cumsum(lens)])
        for P in range(1, n + 1):
            got = O.band_nnz_parts(rp, P)
            nnz = rp[-1]
            want = [0]
            for k in range(1, P):
                want.append(next(r for r in range(n + 1) if P * rp[r] >= k * nnz))
            want.append(n)
            assert list(got) == want
    # uniform rows: boundaries are ceil(k n / P)
    rp = np.arange(0, 7 * 100 + 1, 7)
    assert list(O.band_nnz_parts(rp, 8)) == [-(-k * 100 // 8) for k in range(9)]


def test_substructure_interface_count_closed_form():
    # one separator plane per cut: interface = g^3 - (g - p + 1)^3 per cube
    for g, p in [(160, 4), (20, 2), (17, 3), (9, 1)]:
        perm, parts = O.substructure((g, g, g), (p, p, p), g ** 3)
        assert parts[-1] - parts[-2] == g ** 3 - (g - p + 1) ** 3
        assert sorted(perm) == list(range(g ** 3)) if g <= 20 else True
    perm, parts = O.substructure((160, 160, 160), (4, 4, 4), 160 ** 3)
    assert parts[-1] - parts[-2] == 226107


def test_substructure_decouples_interiors():
    for grid, sub in [((12, 12, 12), (2, 2, 2)), ((11, 9, 13), (3, 2, 4))]:
        A = W.laplace7(grid)
        perm, parts = O.substructure(grid, sub, A.n)
        assert np.array_equal(np.sort(perm), np.arange(A.n))
        assert O.interiors_decoupled(A.rowptr, A.col, perm, parts)
        # interface-last: the interface holds exactly the nodes on cut planes
        assert np.all(np.diff(perm[parts[-2]:]) > 0)
    F27 = W.fe27_deleted(10, seed=3)
    perm, parts = O.substructure(F27.grid, (2, 3, 2), F27.n, node=F27.node)
    assert O.interiors_decoupled(F27.rowptr, F27.col, perm, parts)
    # a wrong grid descriptor couples interiors
    A = W.laplace7((12, 12, 12))
    perm, parts = O.substructure((6, 24, 12), (2, 2, 2), A.n)
    assert not O.interiors_decoupled(A.rowptr, A.col, perm, parts)


def test_partitioned_sweep_is_splitting_independent():
    """Synchronous iterates do not depend on the splitting (the band-row
    iteration counts are identical for every #p in the paper's tables)."""
    A = W.fe27_deleted(9, seed=2)
    xs, b = W.solution_and_rhs(A, 4)
    x = np.zeros(A.n)
    splits = []
    for P in (1, 3, 7):
        splits.append((O.band_row_parts(A.n, P), np.arange(A.n)))
        splits.append((O.band_nnz_parts(A.rowptr, P), np.arange(A.n)))
    perm, parts = O.substructure(A.grid, (2, 2, 2), A.n, node=A.node)
    splits.append((parts, perm))
    for k in range(5):
        y_ref, ss_ref, mx_ref = O.sweep(A, b, x)
        for parts, rows in splits:
            recv, _ = O.dependency_lists(A.rowptr, A.col, parts, rows)
            hp, h = O.halo_of(recv)
            y, ss, mx = O.partitioned_sweep(A, b, x, parts, rows, hp, h)
            assert np.array_equal(y, y_ref)
            assert mx == mx_ref
            assert ss == pytest.approx(ss_ref, rel=1e-13)
        x = y_ref


# ------------------------------------------------------------ the sweep ----

def test_solution_is_fixed_point_nonsymmetric():
    """x* = A^{-1} b (dense LU) is a fixed point of the sweep and has ~0 residual;
    a transposed operand or a dropped term would move it."""
    for seed in range(3):
        A = W.random_dominant(120, seed=seed, density=0.08)
        dense = A.scipy().toarray()
        assert not np.allclose(dense, dense.T)
        b = np.random.default_rng(seed).uniform(-1, 1, 120)
        xs = np.linalg.solve(dense, b)
        y, ss, mx, r = O.sweep(A, b, xs, want_r=True)
        np.testing.assert_allclose(y, xs, rtol=0, atol=1e-13)
        assert np.sqrt(ss) < 1e-12 and mx < 1e-12
        # the residual output is b - A x for any x
        x = np.random.default_rng(seed + 9).uniform(-1, 1, 120)
        _, _, _, r = O.sweep(A, b, x, want_r=True)
        np.testing.assert_allclose(r, b - dense @ x, rtol=0, atol=1e-12)


def test_converged_solve_matches_lu():
    A = W.convection7(6, peclet=0.7)
    dense = A.scipy().toarray()
    b = np.random.default_rng(3).uniform(-1, 1, A.n)
    x, k, rel, st = O.solve(A, b, tol=1e-14, maxit=20000)
    assert st == O.JO_OK and rel <= 1e-14
    xs = np.linalg.solve(dense, b)
    assert np.linalg.norm(x - xs) / np.linalg.norm(xs) < 1e-12


@pytest.mark.parametrize("grid,seed,tol", [((16, 16, 16), 0, 1e-6), ((7, 9, 11), 3, 1e-10), ((5, 5, 5), 1, 1e-12)])
def test_laplace_residual_history_matches_dst_closed_form(grid, seed, tol):
    A = W.laplace7(grid)
    xs, b = W.solution_and_rhs(A, seed)
    x, k, rel, st, hist = O.solve(A, b, tol=tol, maxit=20000, history=True)
    cf = _dst_history(grid, xs, k + 1)
    assert np.all(np.abs(hist - cf) <= 1e-9 * cf + 1e-14)
    # the closed form gives the same stopping sweep
    assert cf[k] <= tol and cf[k - 1] > tol


def test_sweeps_to_1e6_on_16cubed_seed0():
    """637 sweeps to relative residual 1e-6 at 16^3 (numpy seed 0), the count the
    closed form gives; seeds 1 and 2 give 566 and 560."""
    A = W.laplace7(16)
    for seed, want in [(0, 637), (1, 566), (2, 560)]:
        xs, b = W.solution_and_rhs(A, seed)
        _, k, rel, st = O.solve(A, b, tol=1e-6, maxit=5000)
        assert k == want
        cf = _dst_history((16, 16, 16), xs, want + 1)
        assert cf[want] <= 1e-6 < cf[want - 1]


def _dst_crossing(grid, xstar, tol):
    """First k with closed-form relres_k <= tol (bisection; the history is
    monotone for the 7-point Laplacian, whose Jacobi eigenvalues have |mu| < 1),
    with the relative margins of relres_k and relres_{k-1} from tol."""
    gx, gy, gz = grid
    z = F.dstn(xstar.reshape(gz, gy, gx), type=1, norm="ortho")
    ev = [2.0 - 2.0 * np.cos(np.pi * np.arange(1, g + 1) / (g + 1)) for g in (gz, gy, gx)]
    lam = ev[0][:, None, None] + ev[1][None, :, None] + ev[2][None, None, :]
    w = (lam * z) ** 2
    lmu2 = 2.0 * np.log(np.abs(1.0 - lam / 6.0))
    bn = np.sqrt(np.sum(w))
    rel = lambda k: np.sqrt(np.sum(w * np.exp(k * lmu2))) / bn
    lo, hi = 0, 1
    while rel(hi) > tol:
        lo, hi = hi, hi * 2
    while hi - lo > 1:
        mid = (lo + hi) // 2
        lo, hi = (lo, mid) if rel(mid) <= tol else (mid, hi)
    return hi, 1.0 - rel(hi) / tol, rel(hi - 1) / tol - 1.0


def test_160cubed_benchmark_workload_closed_form_and_oracle_sweeps():
    """The benchmark's 160^3 system (numpy seed 0): the closed form reaches
    relres 1e-8 after 42,745 sweeps, with a margin far above rounding on both
    sides of the crossing, so an FP64 solve must stop there exactly; the oracle's
    first sweeps at this size follow the closed form."""
    grid = (160, 160, 160)
    A = W.laplace7(160)
    xs, b = W.solution_and_rhs(A, 0)
    k, below, above = _dst_crossing(grid, xs, 1e-8)
    assert k == 42745
    assert below > 1e-5 and above > 1e-5
    x, kk, rel, st, hist = O.solve(A, b, tol=1e-8, maxit=6, history=True)
    assert st == O.JO_ENOTCONV and len(hist) == 7
    cf = _dst_history(grid, xs, 7)
    assert np.all(np.abs(hist - cf) <= 1e-12 * cf)


def test_asymptotic_contraction_is_spectral_radius():
    """Late residual contraction equals rho(I - D^{-1}A) = cos(pi/(m+1))
    (Sec. 3, convergence theorem; the rate bound (rho+eps)^k)."""
    for m in (10, 16):
        A = W.laplace7(m)
        xs, b = W.solution_and_rhs(A, 7)
        _, k, rel, st, hist = O.solve(A, b, tol=1e-11, maxit=20000, history=True)
        ratio = hist[-1] / hist[-2]
        assert abs(ratio - np.cos(np.pi / (m + 1))) < 1e-6


def test_divergence_when_spectral_radius_exceeds_one():
    """Sec. 3 theorem: the iteration converges iff rho(T) < 1."""
    rng = np.random.default_rng(11)
    n = 30
    for margin, converges in [(0.3, True), (-0.6, False)]:
        M = rng.uniform(-1, 1, (n, n)) * (rng.random((n, n)) < 0.3)
        np.fill_diagonal(M, 0.0)
        M = M + M.T
        np.fill_diagonal(M, (1 + margin) * np.abs(M).sum(axis=1) + 1e-3)
        D = np.diag(np.diag(M))
        rho = max(abs(np.linalg.eigvals(np.linalg.solve(D, D - M))))
        assert (rho < 1) == converges
        A = W.dense_to_csr(M)
        b = rng.uniform(-1, 1, n)
        _, k, rel, st = O.solve(A, b, tol=1e-10, maxit=3000)
        assert (st == O.JO_OK) == converges


def test_multi_rhs_sweep_equals_columnwise():
    A = W.diffusion7(5, seed=2)
    rng = np.random.default_rng(0)
    b = rng.uniform(-1, 1, (A.n, 4))
    x = rng.uniform(-1, 1, (A.n, 4))
    y, ss, mx = O.sweep_multi(A, b, x)
    for c in range(4):
        yc, ssc, mxc = O.sweep(A, b[:, c], x[:, c])
        assert np.array_equal(y[:, c], yc)
        assert ss[c] == ssc and mx[c] == mxc


def test_zero_diagonal_is_rejected():
    M = np.array([[1.0, 2.0], [3.0, 0.0]])
    with pytest.raises(ZeroDivisionError):
        O.solve(W.dense_to_csr(M), np.ones(2))


# ------------------------------------------------- the paper's own counts --

def _paper_counts():
    out = []
    for line in open(golden_path("paper_iteration_counts.txt")):
        line = line.split("#")[0].strip()
        if line:
            N, it = line.split()
            out.append((int(N), int(it)))
    return out


@pytest.mark.parametrize("N,iters", _paper_counts())
def test_q1_laplace_reproduces_paper_iteration_count(N, iters):
    """Q1 FE Laplace on N^3 nodes, b = M_h cos(x+y), stop at ||r||_inf < 1e-8:
    Algorithm 1 counts k+1 iterations (its counter is bumped before the break)."""
    A, b = W.q1_laplace(N)
    x, k, rel, st = O.solve(A, b, tol=1e-8, norm=0, maxit=10000)
    assert st == O.JO_OK
    assert k + 1 == iters


# ------------------------------------------------------------- adjoint -----

def test_adjoint_gradients_match_dense_reference():
    A = W.convection7(4, peclet=0.8)              # non-symmetric: exercises A^T
    dense = A.scipy().toarray()
    rng = np.random.default_rng(2)
    b = rng.uniform(-1, 1, A.n)
    xt = rng.uniform(-1, 1, A.n)
    x, k, rel, st = O.solve(A, b, tol=1e-15, maxit=50000)
    g = 2.0 * (x - xt)
    dA, db, k2, rel2, st2 = O.adjoint_gradients(A, x, g, tol=1e-15, maxit=50000)
    lam = np.linalg.solve(dense.T, g)
    np.testing.assert_allclose(db, lam, rtol=0, atol=1e-11 * np.abs(lam).max())
    rp = A.rowptr.astype(np.int64)
    rowid = np.repeat(np.arange(A.n), np.diff(rp))
    np.testing.assert_allclose(dA, -lam[rowid] * x[A.col], rtol=0, atol=1e-11)
    # central finite differences of L(b, A) = ||A^{-1} b - xt||^2 on a few entries
    L = lambda M, bb: np.sum((np.linalg.solve(M, bb) - xt) ** 2)
    h = 1e-6
    for e in rng.choice(A.nnz, 6, replace=False):
        i, j = rowid[e], A.col[e]
        Mp, Mm = dense.copy(), dense.copy()
        Mp[i, j] += h
        Mm[i, j] -= h
        fd = (L(Mp, b) - L(Mm, b)) / (2 * h)
        assert fd == pytest.approx(dA[e], rel=1e-5, abs=1e-9)
    for i in rng.choice(A.n, 4, replace=False):
        bp, bm = b.copy(), b.copy()
        bp[i] += h
        bm[i] -= h
        fd = (L(dense, bp) - L(dense, bm)) / (2 * h)
        assert fd == pytest.approx(db[i], rel=1e-5, abs=1e-9)


@pytest.mark.parametrize("m,seed", [(5, 0), (6, 3)])
def test_fe27_operator_bound_and_lu_solution(m, seed):
    """The FE-like 27-point operator has no closed form: pin its structure
    (symmetric, rows of 8 to 27 entries), the Jacobi bound that its relative
    dominance margin gives, rho(D^{-1}(L+U)) <= 1/(1+1e-2), and the oracle's
    converged solve against dense LU."""
    A = W.fe27_deleted(m, seed=seed)
    Ad = A.scipy().toarray()
    assert np.array_equal(Ad, Ad.T)
    lens = np.diff(A.rowptr)
    assert lens.min() >= 8 and lens.max() <= 27
    d = np.diag(Ad)
    T = np.eye(A.n) - Ad / d[:, None]
    rho = np.max(np.abs(np.linalg.eigvals(T)))
    assert rho <= 1.0 / 1.01 + 1e-12
    xs, b = W.solution_and_rhs(A, seed)
    x, k, rel, st = O.solve(A, b, None, tol=1e-13, maxit=100000)
    assert st == O.JO_OK
    assert np.max(np.abs(x - np.linalg.solve(Ad, b))) <= 1e-11 * np.max(np.abs(xs))
