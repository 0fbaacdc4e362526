"""CPU oracle for the partitioned synchronous Jacobi solver.

TEST INFRASTRUCTURE ONLY.  Nothing in the product package imports this
module; only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg
of ``bench.py`` use it.  It shares no code with the CUDA path.

What it holds, each piece following the paper (Ahamed & Magoules, "On the
stability and performance of the solution of sparse linear systems by
partitioned procedures"):

* ``sweep`` / ``solve``   -- Jacobi iteration (Sec. 3, component form of
  x^{k+1} = D^{-1}(b - (L+U) x^k)) and Algorithm 1's loop with the test on the
  residual of the current iterate, in plain C compiled without FMA
  contraction (``jacobi_oracle.c``).
* ``band_row_parts``      -- band-row splitting (Sec. 4.2): P contiguous bands,
  band p holding rows [floor(p n / P), floor((p+1) n / P)); with n = 10, P = 3
  this gives the paper's 3/3/4 example.
* ``band_nnz_parts``      -- band-row splitting balanced by non-zeros (Sec.
  4.2.2, weighted partition with vertex weight = row nnz), kept contiguous:
  boundary k is the first row r with P * IA(r) >= k * nnz.
* ``dependency_lists``    -- the receive and send lists of the sparsity-pattern
  splitting (Sec. 4.2.2, tables of receiving and sending dependencies).
* ``substructure``        -- substructuring (Sec. 4.3): geometric boxes with one
  separator node plane per cut, interiors of subdomain 1..S first and the
  interface block last (the block form of Eq. (4.4)).
* ``partitioned_sweep``   -- one sweep per partition on a private copy of x
  holding only owned and received entries (the CPU stand-in for the MPI
  exchange).
* ``split_prepare`` / ``split_sweep`` / ``split_solve`` -- substructuring with
  the interface block split between subdomains (Sec. 4.3): local matrices
  A_s with A33 = sum_s A33^(s), the two-step product (local sums, then
  assembly at the interface) and the weighted interface dot product.
* ``band_row_sets`` / ``box_row_sets`` / ``solve_local`` -- stopping on
  local convergence (Sec. 3, the parallel form of Algorithm 1): every
  partition tests the residual of the rows it holds (its band, or the nodes
  of its box of cells under substructuring).
* ``adjoint_gradients``   -- dL/db = lambda, dL/dA_ij = -lambda_i x_j with
  A^T lambda = dL/dx, the lambda solve done by the same Jacobi loop.

``sweep_omp`` (``jacobi_omp.c``) is not part of the checker: it is the same
row loop spread over the host's cores with OpenMP, timed by the benchmark as
a multi-core CPU baseline.

Parity pins for every function are in ``tests/test_oracle_*.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from typing import Dict, List, Optional, Sequence, Tuple

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "jacobi_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "libjacobi_oracle.so")
_lock = threading.Lock()
_lib = None

JO_OK, JO_EINVAL, JO_ESINGULAR, JO_ENOTCONV, JO_EHALO = 0, 1, 2, 3, 4


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc (no FMA contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


_SRC_OMP = os.path.join(_HERE, "jacobi_omp.c")
_SO_OMP = os.path.join(_BUILD, "libjacobi_omp.so")
_lib_omp = None


def build_omp(force: bool = False) -> str:
    """Compile the multi-core CPU baseline (OpenMP) with gcc."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO_OMP) or os.path.getmtime(_SO_OMP) < os.path.getmtime(_SRC_OMP):
        tmp = _SO_OMP + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
                               "-o", tmp, _SRC_OMP, "-lm"])
        os.replace(tmp, _SO_OMP)
    return _SO_OMP


def _omp():
    global _lib_omp
    with _lock:
        if _lib_omp is None:
            build_omp()
            L = ctypes.CDLL(_SO_OMP)
            P = ctypes.c_void_p
            L.jo_sweep_omp.argtypes = [ctypes.c_int64, P, P, P, P, P, P, P, P, P, P]
            L.jo_sweep_omp.restype = None
            L.jo_omp_threads.restype = ctypes.c_int
            _lib_omp = L
    return _lib_omp


def omp_threads() -> int:
    """Threads the multi-core baseline uses."""
    return int(_omp().jo_omp_threads())


def sweep_omp(A, b: np.ndarray, x: np.ndarray):
    """The multi-core CPU baseline's sweep (a timing baseline, not a checker):
    returns (x_next, sumsq, maxabs) like ``sweep``."""
    M = _mat(A)
    b = np.ascontiguousarray(b, dtype=np.float64)
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.empty(M.n)
    ss = ctypes.c_double()
    mx = ctypes.c_double()
    _omp().jo_sweep_omp(M.n, _p(M.rowptr), _p(M.col), _p(M.val), _p(M.d), _p(M.dinv), _p(b), _p(x), _p(y),
                        ctypes.byref(ss), ctypes.byref(mx))
    return y, ss.value, mx.value


def _c():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_SO)
            P = ctypes.c_void_p
            i64 = ctypes.c_int64
            L.jo_diag.argtypes = [i64, P, P, P, P, P]
            L.jo_sweep.argtypes = [i64, P, P, P, P, P, P, P, P, P, P, P]
            L.jo_solve.argtypes = [i64, P, P, P, P, P, ctypes.c_double, ctypes.c_int, i64, P, P, P]
            L.jo_partitioned_sweep.argtypes = [i64, P, P, P, P, P, P, P, i64, P, P, P, P, P, P, P]
            L.jo_spmv.argtypes = [i64, P, P, P, P, P]
            L.jo_sweep_multi.argtypes = [i64, i64, P, P, P, P, P, P, P, P, P, P]
            L.jo_split_diag.argtypes = [i64, i64, P, P, P, P, P, P]
            L.jo_split_sweep.argtypes = [i64, P, i64, P, P, P, P, P, P, P, P, P, P, P, P, P]
            for f in (L.jo_diag, L.jo_sweep, L.jo_solve, L.jo_partitioned_sweep, L.jo_sweep_multi,
                      L.jo_split_diag, L.jo_split_sweep):
                f.restype = ctypes.c_int
            L.jo_spmv.restype = None
            _lib = L
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


class _Mat:
    """Oracle-side copy of a CSR matrix (int64 row pointers, int32 columns)."""

    def __init__(self, n, rowptr, col, val):
        self.n = int(n)
        self.rowptr = np.ascontiguousarray(rowptr, dtype=np.int64)
        self.col = np.ascontiguousarray(col, dtype=np.int32)
        self.val = np.ascontiguousarray(val, dtype=np.float64)
        self.d = np.empty(self.n)
        self.dinv = np.empty(self.n)
        st = _c().jo_diag(self.n, _p(self.rowptr), _p(self.col), _p(self.val), _p(self.d), _p(self.dinv))
        if st != JO_OK:
            raise ZeroDivisionError("zero or missing diagonal entry")


def _mat(A) -> _Mat:
    return A if isinstance(A, _Mat) else _Mat(A.n, A.rowptr, A.col, A.val)


def prepare(A) -> _Mat:
    """Precompute D and D^{-1} once (Algorithm 1) for repeated sweeps."""
    return _mat(A)


def sweep(A, b: np.ndarray, x: np.ndarray, want_r: bool = False):
    """One synchronous Jacobi sweep.

    Returns (x_next, sumsq, maxabs[, r]) where sumsq = ||b - A x||_2^2 and
    maxabs = ||b - A x||_inf of the *pre-update* iterate x.
    """
    M = _mat(A)
    b = np.ascontiguousarray(b, dtype=np.float64)
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.empty(M.n)
    r = np.empty(M.n) if want_r else None
    ss = ctypes.c_double()
    mx = ctypes.c_double()
    _c().jo_sweep(M.n, _p(M.rowptr), _p(M.col), _p(M.val), _p(M.d), _p(M.dinv), _p(b), _p(x), _p(y),
                  _p(r) if want_r else None, ctypes.byref(ss), ctypes.byref(mx))
    if want_r:
        return y, ss.value, mx.value, r
    return y, ss.value, mx.value


def sweep_multi(A, b: np.ndarray, x: np.ndarray):
    """Sweep for row-major n x nrhs right-hand sides sharing A."""
    M = _mat(A)
    nrhs = b.shape[1]
    b = np.ascontiguousarray(b, dtype=np.float64)
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.empty_like(x)
    ss = np.empty(nrhs)
    mx = np.empty(nrhs)
    _c().jo_sweep_multi(M.n, nrhs, _p(M.rowptr), _p(M.col), _p(M.val), _p(M.d), _p(M.dinv), _p(b), _p(x),
                        _p(y), _p(ss), _p(mx))
    return y, ss, mx


def solve(A, b: np.ndarray, x0: Optional[np.ndarray] = None, tol: float = 1e-8, maxit: int = 100000,
          norm: int = 2, history: bool = False):
    """Algorithm 1: returns (x_k, k, relres_k, status[, hist]).

    k is the number of updates applied (the paper's iteration count is k+1),
    relres the relative 2-norm (norm=2) or absolute inf-norm (norm=0) of r^k.
    """
    M = _mat(A)
    b = np.ascontiguousarray(b, dtype=np.float64)
    x = np.zeros(M.n) if x0 is None else np.array(x0, dtype=np.float64, copy=True)
    hist = np.empty(maxit + 1) if history else None
    k = ctypes.c_int64()
    rel = ctypes.c_double()
    st = _c().jo_solve(M.n, _p(M.rowptr), _p(M.col), _p(M.val), _p(b), _p(x), float(tol), int(norm),
                       int(maxit), ctypes.byref(k), ctypes.byref(rel), _p(hist) if history else None)
    if st == JO_ESINGULAR:
        raise ZeroDivisionError("zero or missing diagonal entry")
    if st == JO_EINVAL:
        raise ValueError("invalid arguments")
    out = (x, int(k.value), float(rel.value), st)
    if history:
        out = out + (hist[: k.value + 1].copy(),)
    return out


def spmv(A, x: np.ndarray) -> np.ndarray:
    M = _mat(A)
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.empty(M.n)
    _c().jo_spmv(M.n, _p(M.rowptr), _p(M.col), _p(M.val), _p(x), _p(y))
    return y


# ---------------------------------------------------------------------------
# Splittings (Sec. 4) -- integer work, plain numpy
# ---------------------------------------------------------------------------

def band_row_parts(n: int, P: int) -> np.ndarray:
    """Band boundaries: band p = rows [floor(p n / P), floor((p+1) n / P))."""
    if P < 1 or P > max(n, 1):
        raise ValueError("need 1 <= P <= n")
    return np.array([(p * n) // P for p in range(P + 1)], dtype=np.int64)


def band_nnz_parts(rowptr: np.ndarray, P: int) -> np.ndarray:
    """nnz-balanced contiguous bands: boundary k = min{ r : P * IA(r) >= k * nnz }."""
    rp = np.asarray(rowptr, dtype=np.int64)
    n = rp.size - 1
    if P < 1 or P > max(n, 1):
        raise ValueError("need 1 <= P <= n")
    nnz = int(rp[-1])
    out = np.empty(P + 1, dtype=np.int64)
    for k in range(P + 1):
        target = k * nnz
        r = 0
        # first row r with P * rp[r] >= target (bisection over the non-decreasing IA)
        lo, hi = 0, n
        while lo < hi:
            mid = (lo + hi) // 2
            if P * int(rp[mid]) >= target:
                hi = mid
            else:
                lo = mid + 1
        r = lo
        out[k] = r
    out[0], out[P] = 0, n
    return out


def owner_of_rows(part_ptr: np.ndarray, rows: np.ndarray, n: int) -> np.ndarray:
    """owner[i] = partition holding original row i."""
    owner = np.full(n, -1, dtype=np.int64)
    for p in range(len(part_ptr) - 1):
        owner[rows[part_ptr[p]:part_ptr[p + 1]]] = p
    return owner


def dependency_lists(rowptr, col, part_ptr: np.ndarray, rows: Optional[np.ndarray] = None):
    """Receive/send lists of the sparsity-pattern splitting (Sec. 4.2.2).

    ``rows[part_ptr[p]:part_ptr[p+1]]`` are the (original) rows of partition p;
    rows=None means contiguous bands (rows = arange(n)).
    Returns (recv, send): recv[p][q] = sorted original indices of x that p
    receives from q; send[q][p] = recv[p][q].
    """
    rp = np.asarray(rowptr, dtype=np.int64)
    cl = np.asarray(col, dtype=np.int64)
    n = rp.size - 1
    if rows is None:
        rows = np.arange(n, dtype=np.int64)
    owner = owner_of_rows(part_ptr, rows, n)
    P = len(part_ptr) - 1
    recv: List[Dict[int, np.ndarray]] = [dict() for _ in range(P)]
    send: List[Dict[int, np.ndarray]] = [dict() for _ in range(P)]
    for p in range(P):
        prow = rows[part_ptr[p]:part_ptr[p + 1]]
        if prow.size == 0:
            continue
        starts, ends = rp[prow], rp[prow + 1]
        idx = np.concatenate([np.arange(s, e) for s, e in zip(starts, ends)]) if prow.size else np.zeros(0, np.int64)
        cols = np.unique(cl[idx])
        ext = cols[owner[cols] != p]
        for q in np.unique(owner[ext]):
            lst = ext[owner[ext] == q]
            recv[p][int(q)] = lst
            send[int(q)][p] = lst
    return recv, send


def halo_of(recv) -> Tuple[np.ndarray, np.ndarray]:
    """Flatten receive lists into (halo_ptr, halo) for partitioned_sweep."""
    ptr = [0]
    items = []
    for p in range(len(recv)):
        lst = [recv[p][q] for q in sorted(recv[p])]
        h = np.concatenate(lst) if lst else np.zeros(0, np.int64)
        items.append(h)
        ptr.append(ptr[-1] + h.size)
    return np.array(ptr, dtype=np.int64), (np.concatenate(items) if items else np.zeros(0, np.int64)).astype(np.int64)


def substructure(grid: Sequence[int], sub: Sequence[int], n: int, node: Optional[np.ndarray] = None):
    """Geometric substructuring with the interface last (Sec. 4.3).

    The node grid (gx, gy, gz) is cut along each axis at the node planes
    c_t = floor(t g / p), t = 1..p-1; a node on any cut plane belongs to the
    interface.  Every other node belongs to subdomain
    s = sx + px (sy + py sz), sx = number of cuts below its x coordinate.
    New order: interiors of subdomains 0..S-1 (ascending original row within
    each), then the interface (ascending original row).

    Returns (perm, part_ptr): perm[new] = original row; partitions 0..S-1 are
    the interiors, partition S the interface.
    """
    gx, gy, gz = (int(v) for v in grid)
    px, py, pz = (int(v) for v in sub)
    if min(px, py, pz) < 1 or px > gx or py > gy or pz > gz:
        raise ValueError("bad subdomain counts")
    nodes = np.arange(n, dtype=np.int64) if node is None else np.asarray(node, dtype=np.int64)
    X = nodes % gx
    Y = (nodes // gx) % gy
    Z = nodes // (gx * gy)

    def axis(coord, g, p):
        cuts = np.array([(t * g) // p for t in range(1, p)], dtype=np.int64)
        on = np.isin(coord, cuts)
        s = np.searchsorted(cuts, coord, side="left")  # number of cuts strictly below coord
        return on, s

    onx, sx = axis(X, gx, px)
    ony, sy = axis(Y, gy, py)
    onz, sz = axis(Z, gz, pz)
    iface = onx | ony | onz
    S = px * py * pz
    sid = np.where(iface, S, sx + px * (sy + py * sz))
    perm = np.argsort(sid, kind="stable").astype(np.int64)
    counts = np.bincount(sid, minlength=S + 1)
    part_ptr = np.zeros(S + 2, dtype=np.int64)
    np.cumsum(counts, out=part_ptr[1:])
    return perm, part_ptr


def interiors_decoupled(rowptr, col, perm: np.ndarray, part_ptr: np.ndarray) -> bool:
    """True when no entry couples the interiors of two different subdomains
    (the zero blocks of Eq. (4.4))."""
    n = len(rowptr) - 1
    S = len(part_ptr) - 2
    sid = np.empty(n, dtype=np.int64)
    for p in range(S + 1):
        sid[perm[part_ptr[p]:part_ptr[p + 1]]] = p
    rp = np.asarray(rowptr, dtype=np.int64)
    rowid = np.repeat(np.arange(n), np.diff(rp))
    a, b = sid[rowid], sid[np.asarray(col, dtype=np.int64)]
    bad = (a != b) & (a < S) & (b < S)
    return not bool(bad.any())


def partitioned_sweep(A, b: np.ndarray, x: np.ndarray, part_ptr: np.ndarray, rows: np.ndarray,
                      halo_ptr: np.ndarray, halo: np.ndarray):
    """One sweep with each partition restricted to its owned and received x."""
    M = _mat(A)
    b = np.ascontiguousarray(b, dtype=np.float64)
    x = np.ascontiguousarray(x, dtype=np.float64)
    part_ptr = np.ascontiguousarray(part_ptr, dtype=np.int64)
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    halo_ptr = np.ascontiguousarray(halo_ptr, dtype=np.int64)
    halo = np.ascontiguousarray(halo, dtype=np.int64)
    y = np.full(M.n, np.nan)
    ss = ctypes.c_double()
    mx = ctypes.c_double()
    st = _c().jo_partitioned_sweep(M.n, _p(M.rowptr), _p(M.col), _p(M.val), _p(M.d), _p(M.dinv), _p(b), _p(x),
                                   len(part_ptr) - 1, _p(part_ptr), _p(rows), _p(halo_ptr), _p(halo), _p(y),
                                   ctypes.byref(ss), ctypes.byref(mx))
    if st == JO_EHALO:
        raise LookupError("a row read an x entry missing from its dependency list")
    return y, ss.value, mx.value


# ---------------------------------------------------------------------------
# Substructuring with the interface block split between subdomains (Sec. 4.3)
# ---------------------------------------------------------------------------

class _Split:
    """Local matrices of all subdomains stacked in subdomain order, with
    global columns, and the assembled diagonal (computed once)."""

    def __init__(self, locals_, n: int):
        self.n = int(n)
        self.nsub = len(locals_)
        ptr, rows, cols, vals, grow = [0], [np.zeros(1, np.int64)], [], [], []
        for L in locals_:
            l2g = np.asarray(L.l2g, dtype=np.int64)
            rp = np.asarray(L.rowptr, dtype=np.int64)
            rows.append(rows[-1][-1] + rp[1:])
            cols.append(l2g[np.asarray(L.col, dtype=np.int64)])
            vals.append(np.asarray(L.val, dtype=np.float64))
            grow.append(l2g)
            ptr.append(ptr[-1] + L.n)
        self.sub_ptr = np.array(ptr, dtype=np.int64)
        self.rowptr = np.ascontiguousarray(np.concatenate(rows), dtype=np.int64)
        self.gcol = np.ascontiguousarray(np.concatenate(cols) if cols else np.zeros(0), dtype=np.int32)
        self.val = np.ascontiguousarray(np.concatenate(vals) if vals else np.zeros(0), dtype=np.float64)
        self.grow = np.ascontiguousarray(np.concatenate(grow) if grow else np.zeros(0), dtype=np.int32)
        self.mult = np.bincount(self.grow, minlength=self.n).astype(np.int32)
        if (self.mult == 0).any():
            raise ValueError("a node belongs to no subdomain")
        self.d = np.empty(self.n)
        self.dinv = np.empty(self.n)
        st = _c().jo_split_diag(int(self.sub_ptr[-1]), self.n, _p(self.rowptr), _p(self.gcol), _p(self.val),
                                _p(self.grow), _p(self.d), _p(self.dinv))
        if st != JO_OK:
            raise ZeroDivisionError("zero assembled diagonal entry")

    def interface(self) -> np.ndarray:
        """Global nodes held by two or more subdomains (the interface set)."""
        return np.flatnonzero(self.mult >= 2)


def split_prepare(locals_, n: int) -> _Split:
    """Stack the local matrices (each with ``n``, ``rowptr``, ``col``, ``val``,
    ``l2g``) and assemble the diagonal once."""
    return _Split(locals_, n)


def split_sweep(P: _Split, b: np.ndarray, x: np.ndarray, want_r: bool = False):
    """One Jacobi sweep in the split form: local off-diagonal sums per
    subdomain, assembly at the interface in subdomain order, the update with
    the assembled diagonal, and the weighted interface dot product.

    Returns (x_next, sumsq, maxabs[, r]) of the pre-update iterate x."""
    b = np.ascontiguousarray(b, dtype=np.float64)
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.empty(P.n)
    r = np.empty(P.n) if want_r else None
    ss = ctypes.c_double()
    mx = ctypes.c_double()
    _c().jo_split_sweep(P.nsub, _p(P.sub_ptr), P.n, _p(P.rowptr), _p(P.gcol), _p(P.val), _p(P.grow),
                        _p(P.mult), _p(P.d), _p(P.dinv), _p(b), _p(x), _p(y), _p(r) if want_r else None,
                        ctypes.byref(ss), ctypes.byref(mx))
    if want_r:
        return y, ss.value, mx.value, r
    return y, ss.value, mx.value


def split_solve(P: _Split, b: np.ndarray, x0: Optional[np.ndarray] = None, tol: float = 1e-8,
                maxit: int = 100000, norm: int = 2):
    """Algorithm 1 over split sweeps: returns (x_k, k, relres_k, status) with
    the same test and counting as ``solve``."""
    b = np.ascontiguousarray(b, dtype=np.float64)
    x = np.zeros(P.n) if x0 is None else np.array(x0, dtype=np.float64, copy=True)
    bnorm = float(np.sqrt(np.sum(b * b)))
    k = 0
    while True:
        y, ss, mx = split_sweep(P, b, x)
        if norm == 2:
            rel = np.sqrt(ss) / bnorm if bnorm > 0 else np.sqrt(ss)
        else:
            rel = mx
        if rel <= tol:
            return x, k, float(rel), JO_OK
        if k == maxit:
            return x, k, float(rel), JO_ENOTCONV
        x = y
        k += 1


# ---------------------------------------------------------------------------
# Adjoint (gradients through the solve)
# ---------------------------------------------------------------------------

# ---------------------------------------------------------------------------
# Stopping on local convergence (Sec. 3, the parallel form of Algorithm 1)
# ---------------------------------------------------------------------------

def band_row_sets(part_ptr: np.ndarray) -> List[np.ndarray]:
    """Rows each band-row partition holds (Sec. 4.2): its band, in the
    original numbering (band splittings do not reorder rows)."""
    pp = np.asarray(part_ptr, dtype=np.int64)
    return [np.arange(pp[q], pp[q + 1], dtype=np.int64) for q in range(len(pp) - 1)]


def box_row_sets(grid: Sequence[int], sub: Sequence[int], n: int,
                 node: Optional[np.ndarray] = None) -> List[np.ndarray]:
    """Rows each subdomain of the geometric substructuring holds (Sec. 4.3):
    the nodes of its box of grid cells, i.e. its interior nodes and the
    interface nodes on its box's boundary.

    Built from the cells: along an axis of g nodes cut into p parts (cut node
    planes c_t = floor(t g / p), t = 1..p-1), the cells have lower corners
    -1..g-1 (the outer layer touches the Dirichlet boundary) and box t holds
    the cells whose lower corner lies in [c_t, c_{t+1}) with c_0 = -1 and
    c_p = g; a node belongs to a box when it is a corner of one of its cells.
    Returns one array of rows (ascending) per subdomain
    s = sx + px (sy + py sz)."""
    gx, gy, gz = (int(v) for v in grid)
    px, py, pz = (int(v) for v in sub)
    nodes = np.arange(n, dtype=np.int64) if node is None else np.asarray(node, dtype=np.int64)
    row_of = np.full(gx * gy * gz, -1, dtype=np.int64)
    row_of[nodes] = np.arange(n, dtype=np.int64)

    def cell_ranges(g, p):
        c = [-1] + [(t * g) // p for t in range(1, p)] + [g]
        return [(c[t], c[t + 1]) for t in range(p)]

    out = []
    for sz, (z0, z1) in enumerate(cell_ranges(gz, pz)):
        for sy, (y0, y1) in enumerate(cell_ranges(gy, py)):
            for sx, (x0, x1) in enumerate(cell_ranges(gx, px)):
                keep = set()
                for cz in range(z0, z1):
                    for cy in range(y0, y1):
                        for cx in range(x0, x1):
                            for dz in (0, 1):
                                for dy in (0, 1):
                                    for dx in (0, 1):
                                        i, j, k = cx + dx, cy + dy, cz + dz
                                        if 0 <= i < gx and 0 <= j < gy and 0 <= k < gz:
                                            r = row_of[i + gx * (j + gy * k)]
                                            if r >= 0:
                                                keep.add(int(r))
                out.append(np.array(sorted(keep), dtype=np.int64))
    return out


def solve_local(A, b: np.ndarray, sets: Sequence[np.ndarray], x0: Optional[np.ndarray] = None,
                tol: float = 1e-8, maxit: int = 100000, rule: str = "first"):
    """Algorithm 1 with the convergence test made per partition.

    Partition p's local test at iterate x^k is max_{i in sets[p]} |r_i| <= tol
    with r = b - A x^k (the experiments' infinity-norm criterion, Sec. 5.2,
    restricted to the rows the partition holds).  rule "all": stop at the
    first k at which every partition passes at once (with the infinity norm
    this is the global test); rule "first": stop at the first k at which some
    partition passes.  Sets must be non-empty.

    Returns (x_k, k, p, local_p, status): p is the lowest-numbered partition
    with the smallest local value at the stopping iterate (rule "first") or
    the one with the largest (rule "all"), local_p that value; status as in
    ``solve``."""
    M = _mat(A)
    b = np.ascontiguousarray(b, dtype=np.float64)
    x = np.zeros(M.n) if x0 is None else np.array(x0, dtype=np.float64, copy=True)
    sets = [np.asarray(S, dtype=np.int64) for S in sets]
    if not sets or any(len(S) == 0 for S in sets):
        raise ValueError("every partition must hold rows")
    k = 0
    while True:
        y, ss, mx, r = sweep(M, b, x, want_r=True)
        loc = np.array([np.max(np.abs(r[S])) for S in sets])
        loc = np.where(np.isnan(loc), np.inf, loc)
        p = int(np.argmin(loc)) if rule == "first" else int(np.argmax(loc))
        if loc[p] <= tol:
            return x, k, p, float(loc[p]), JO_OK
        if k >= maxit:
            return x, k, p, float(loc[p]), JO_ENOTCONV
        x = y
        k += 1


def transpose(A):
    """A^T in CSR (rows of A^T keep ascending column order)."""
    import scipy.sparse as sp
    S = sp.csr_matrix((np.asarray(A.val), np.asarray(A.col), np.asarray(A.rowptr)), shape=(A.n, A.n))
    T = S.T.tocsr()
    T.sort_indices()
    return _Mat(A.n, T.indptr, T.indices, T.data)


def adjoint_gradients(A, x: np.ndarray, dLdx: np.ndarray, tol: float, maxit: int, norm: int = 2):
    """Solve A^T lambda = dL/dx by the same Jacobi loop, then
    dL/db = lambda and dL/dA_ij = -lambda_i x_j on the pattern of A (stored order).

    Returns (dA_values, db, sweeps, relres, status)."""
    At = transpose(A)
    lam, k, rel, st = solve(At, dLdx, None, tol=tol, maxit=maxit, norm=norm)
    rp = np.asarray(A.rowptr, dtype=np.int64)
    rowid = np.repeat(np.arange(A.n), np.diff(rp))
    dA = -lam[rowid] * np.asarray(x)[np.asarray(A.col, dtype=np.int64)]
    return dA, lam, k, rel, st
