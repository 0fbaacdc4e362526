"""Seeded synthetic inputs for the partitioned Jacobi solver.

This module only *builds inputs*: sparse matrices in CSR form, right-hand
sides and initial guesses, all from numpy's seeded ``default_rng``.  It holds
none of the Jacobi method's arithmetic (no sweep, no residual, no splitting),
so both the CPU oracle and the CUDA path can be fed from it without sharing
any of the method's code.  ``b = A x*`` products are formed with scipy's
sparse matrix-vector product as part of the input recipe.

Matrices (the paper's experiments use finite-element Laplace matrices, Sec. 5.1;
those files are not available, so these synthetic families stand in for them):

* ``laplace7``        -- 7-point finite-difference Laplacian on a gx*gy*gz grid of
                         interior nodes, homogeneous Dirichlet boundary
                         (diagonal 6, off-diagonal -1).
* ``diffusion7``      -- variable-coefficient 7-point diffusion, log-normal edge
                         conductivities (boundary edges included).
* ``fe27_deleted``    -- FE-like 27-point hexahedral operator: element matrices
                         c_e (8 I - 1 1^T) on the surviving elements of an
                         m^3-node grid, diagonal set to (1+margin) times the
                         off-diagonal row sum.
* ``q1_laplace``      -- trilinear (Q1) finite-element Laplacian on the unit cube
                         with Dirichlet nodes removed and b = M_h f,
                         f = cos(x + y) (the paper's Set-1 problem, Sec. 5.1.1).
* ``convection7``     -- small non-symmetric 7-point operator (diffusion plus
                         first-order upwind convection), used to exercise A^T.
* ``random_irregular`` -- unstructured diagonally dominant matrix with an
                         irregular row-length mix (a few rows longer than a
                         staged tile), entries in random column order.
* ``cell_box_locals``  -- the local matrices of substructuring with the
                         interface block split between subdomains (Sec. 4.3):
                         each subdomain assembles ``laplace7`` or ``q1_laplace``
                         from its own box of grid cells only.
* ``paper_csr_example`` / ``paper_pattern_10x10`` -- the small matrices printed
                         in the paper (Sec. 4.1 CSR example, Sec. 4.2.2 three-band
                         example).

Every matrix is returned as a :class:`CSR` whose rows keep their entries in
ascending column order (``random_irregular`` excepted: its rows are shuffled,
to exercise the stored-order summation).  Row ``r`` of a grid matrix sits at grid node
``node[r]`` (``i + gx*(j + gy*k)``); ``node is None`` means the natural
ordering ``node[r] == r``.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import Optional, Tuple

import numpy as np
import scipy.sparse as sp


@dataclass
class CSR:
    """A square sparse matrix in 0-based CSR form (int32 indices, float64 values)."""

    n: int
    rowptr: np.ndarray            # int32[n+1]
    col: np.ndarray               # int32[nnz]
    val: np.ndarray               # float64[nnz]
    grid: Optional[Tuple[int, int, int]] = None   # (gx, gy, gz) of the node grid
    node: Optional[np.ndarray] = None             # int64[n] grid node of each row
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def nnz(self) -> int:
        return int(self.rowptr[-1])

    def scipy(self) -> sp.csr_matrix:
        """A scipy copy.  The arrays are copied: scipy canonicalises a matrix
        in place (sorts each row's columns), which would change the stored
        entry order of this CSR and with it the order of every row's sum."""
        return sp.csr_matrix((self.val.copy(), self.col.copy(), self.rowptr.copy()), shape=(self.n, self.n))

    def stats(self) -> dict:
        """Matrix statistics in the columns the paper tabulates (Sec. 5.1.3)."""
        lens = np.diff(self.rowptr.astype(np.int64))
        rows = np.repeat(np.arange(self.n, dtype=np.int64), lens)
        band = int(np.max(self.col.astype(np.int64) - rows)) if self.nnz else 0
        return {
            "h": self.n,
            "nnz": self.nnz,
            "density_pct": 100.0 * self.nnz / float(self.n) ** 2,
            "bandwidth": band,
            "max_row": int(lens.max()) if self.n else 0,
            "nnz_per_row": self.nnz / self.n if self.n else 0.0,
            "nnz_per_row_std": float(lens.std()) if self.n else 0.0,
        }


def _rows_to_csr(n: int, cols: np.ndarray, vals: np.ndarray, mask: np.ndarray) -> Tuple[np.ndarray, np.ndarray, np.ndarray]:
    """Flatten per-row slot tables (n x S, slots already in column order) into CSR."""
    counts = mask.sum(axis=1).astype(np.int64)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])
    if rowptr[-1] >= 2**31:
        raise ValueError("matrix too large for int32 indices")
    col = cols[mask].astype(np.int32)
    val = vals[mask].astype(np.float64)
    return rowptr.astype(np.int32), col, val


# ---------------------------------------------------------------------------
# 7-point operators
# ---------------------------------------------------------------------------

_OFF7 = [(0, 0, -1), (0, -1, 0), (-1, 0, 0), (0, 0, 0), (1, 0, 0), (0, 1, 0), (0, 0, 1)]  # (dx,dy,dz), column order


def _grid_dims(m) -> Tuple[int, int, int]:
    if isinstance(m, (tuple, list)):
        gx, gy, gz = (int(v) for v in m)
    else:
        gx = gy = gz = int(m)
    if min(gx, gy, gz) < 1:
        raise ValueError("grid dimensions must be >= 1")
    return gx, gy, gz


def _stencil7(gx: int, gy: int, gz: int, offdiag: dict, diag: np.ndarray, name: str) -> CSR:
    """Assemble a 7-point operator from per-direction coupling arrays.

    ``offdiag[(dx,dy,dz)]`` is an array shaped (gz,gy,gx) holding a(p, p+d)
    (ignored where p+d leaves the grid); ``diag`` is shaped (gz,gy,gx).
    """
    n = gx * gy * gz
    k, j, i = np.meshgrid(np.arange(gz), np.arange(gy), np.arange(gx), indexing="ij")
    cols = np.empty((n, 7), dtype=np.int64)
    vals = np.empty((n, 7), dtype=np.float64)
    mask = np.empty((n, 7), dtype=bool)
    lin = (i + gx * (j + gy * k)).ravel()
    for s, (dx, dy, dz) in enumerate(_OFF7):
        ii, jj, kk = i + dx, j + dy, k + dz
        ok = (ii >= 0) & (ii < gx) & (jj >= 0) & (jj < gy) & (kk >= 0) & (kk < gz)
        cols[:, s] = lin + dx + gx * (dy + gy * dz)
        if (dx, dy, dz) == (0, 0, 0):
            vals[:, s] = diag.ravel()
        else:
            vals[:, s] = offdiag[(dx, dy, dz)].ravel()
        mask[:, s] = ok.ravel()
    rowptr, col, val = _rows_to_csr(n, cols, vals, mask)
    return CSR(n, rowptr, col, val, grid=(gx, gy, gz), node=None, name=name)


def laplace7(m) -> CSR:
    """7-point Laplacian on an m^3 (or gx*gy*gz) interior grid, Dirichlet boundary.

    Diagonal 6, off-diagonal -1; nnz = 7 m^3 - 6 m^2 for a cube.
    """
    gx, gy, gz = _grid_dims(m)
    shape = (gz, gy, gx)
    off = {d: np.full(shape, -1.0) for d in _OFF7 if d != (0, 0, 0)}
    A = _stencil7(gx, gy, gz, off, np.full(shape, 6.0), name=f"laplace7_{gx}x{gy}x{gz}")
    return A


def diffusion7(m, seed: int, sigma: float = 1.0) -> CSR:
    """Variable-coefficient 7-point diffusion with log-normal edge conductivities.

    Every grid edge, including the edges from boundary nodes to the Dirichlet
    boundary, carries sigma_e = exp(N(0, sigma^2)).  a_ij = -sigma_ij and
    a_ii = sum of the six incident conductivities (symmetric, strictly
    diagonally dominant on boundary rows, weakly elsewhere).
    """
    gx, gy, gz = _grid_dims(m)
    rng = np.random.default_rng(seed)
    # conductivity of the edge between node p-1 and p along each axis (index p along that axis, 0..g)
    ex = np.exp(sigma * rng.standard_normal((gz, gy, gx + 1)))
    ey = np.exp(sigma * rng.standard_normal((gz, gy + 1, gx)))
    ez = np.exp(sigma * rng.standard_normal((gz + 1, gy, gx)))
    off = {
        (-1, 0, 0): -ex[:, :, :-1], (1, 0, 0): -ex[:, :, 1:],
        (0, -1, 0): -ey[:, :-1, :], (0, 1, 0): -ey[:, 1:, :],
        (0, 0, -1): -ez[:-1, :, :], (0, 0, 1): -ez[1:, :, :],
    }
    diag = ex[:, :, :-1] + ex[:, :, 1:] + ey[:, :-1, :] + ey[:, 1:, :] + ez[:-1, :, :] + ez[1:, :, :]
    return _stencil7(gx, gy, gz, off, diag, name=f"diffusion7_{gx}x{gy}x{gz}_s{seed}")


def convection7(m, peclet: float = 0.5) -> CSR:
    """Non-symmetric 7-point operator: Laplacian plus first-order upwind convection.

    Convection along +x with cell Peclet number ``peclet`` adds -peclet to the
    (i-1) coupling and +peclet to the diagonal, so A != A^T while the matrix
    stays diagonally dominant.
    """
    gx, gy, gz = _grid_dims(m)
    shape = (gz, gy, gx)
    off = {d: np.full(shape, -1.0) for d in _OFF7 if d != (0, 0, 0)}
    off[(-1, 0, 0)] = np.full(shape, -1.0 - peclet)
    return _stencil7(gx, gy, gz, off, np.full(shape, 6.0 + peclet), name=f"convection7_{gx}")


# ---------------------------------------------------------------------------
# 27-point operators
# ---------------------------------------------------------------------------

def _offsets27_sorted(gx: int, gy: int):
    offs = [(dx, dy, dz) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]
    return sorted(offs, key=lambda d: d[0] + gx * (d[1] + gy * d[2]))


def _shared_element_sum(ce: np.ndarray, d, nshape) -> np.ndarray:
    """For every node p, sum of element weights ``ce`` over the hex elements that
    contain both p and p+d.  ``ce`` is shaped (gz-1, gy-1, gx-1)."""
    gz, gy, gx = nshape
    pad = np.zeros((gz + 1, gy + 1, gx + 1))
    pad[1:gz, 1:gy, 1:gx] = ce          # element (ez,ey,ex) with lower corner node (ez,ey,ex) sits at pad[ez+1,ey+1,ex+1]
    out = np.zeros(nshape)
    # element lower corner along an axis: d=0 -> p-1 or p ; d=+1 -> p ; d=-1 -> p-1
    choices = []
    for dd in (d[2], d[1], d[0]):
        choices.append((-1, 0) if dd == 0 else ((0,) if dd == 1 else (-1,)))
    for oz in choices[0]:
        for oy in choices[1]:
            for ox in choices[2]:
                out += pad[1 + oz:1 + oz + gz, 1 + oy:1 + oy + gy, 1 + ox:1 + ox + gx]
    return out


def fe27_deleted(m: int, seed: int, delete_frac: float = 0.10, margin: float = 1e-2,
                 cmin: float = 0.1, cmax: float = 10.0) -> CSR:
    """FE-like 27-point hexahedral operator with randomly deleted elements.

    m^3 nodes, (m-1)^3 hex elements; round(delete_frac * ne) elements removed
    (uniform random choice); the rest carry c_e = exp(U[ln cmin, ln cmax]) and
    the element matrix c_e (8 I_8 - 1 1^T), i.e. each element couples its 8
    nodes pairwise with weight -c_e.  After assembly the diagonal is set to
    (1 + margin) * sum_{j != i} |a_ij| (strict dominance by a relative margin),
    and nodes touching no surviving element are dropped.  Rows hold 8..27
    entries.
    """
    gx = gy = gz = int(m)
    ne = (m - 1) ** 3
    rng = np.random.default_rng(seed)
    c = np.exp(rng.uniform(math.log(cmin), math.log(cmax), size=ne))
    dele = rng.choice(ne, size=int(round(delete_frac * ne)), replace=False)
    alive = np.ones(ne, dtype=bool)
    alive[dele] = False
    ce = (c * alive).reshape(m - 1, m - 1, m - 1)
    nshape = (gz, gy, gx)
    # nodes that touch a surviving element
    touch = _shared_element_sum(alive.reshape(m - 1, m - 1, m - 1).astype(np.float64), (0, 0, 0), nshape) > 0
    keep = touch.ravel()
    n = int(keep.sum())
    node_of_row = np.nonzero(keep)[0].astype(np.int64)
    row_of_node = np.full(gx * gy * gz, -1, dtype=np.int64)
    row_of_node[node_of_row] = np.arange(n, dtype=np.int64)

    k, j, i = np.meshgrid(np.arange(gz), np.arange(gy), np.arange(gx), indexing="ij")
    offs = _offsets27_sorted(gx, gy)
    cols = np.empty((n, 27), dtype=np.int64)
    vals = np.empty((n, 27), dtype=np.float64)
    mask = np.empty((n, 27), dtype=bool)
    rowsum = np.zeros(n)
    diag_slot = None
    for s, d in enumerate(offs):
        if d == (0, 0, 0):
            diag_slot = s
            continue
        w = _shared_element_sum(ce, d, nshape).ravel()[keep]
        ii, jj, kk = i + d[0], j + d[1], k + d[2]
        inside = ((ii >= 0) & (ii < gx) & (jj >= 0) & (jj < gy) & (kk >= 0) & (kk < gz)).ravel()[keep]
        nb = (node_of_row + d[0] + gx * (d[1] + gy * d[2]))
        nb = np.where(inside, nb, 0)
        ok = inside & (w > 0)
        cols[:, s] = np.where(ok, row_of_node[nb], 0)
        vals[:, s] = -w
        mask[:, s] = ok
        rowsum += np.where(ok, w, 0.0)
    cols[:, diag_slot] = np.arange(n)
    vals[:, diag_slot] = (1.0 + margin) * rowsum
    mask[:, diag_slot] = True
    rowptr, col, val = _rows_to_csr(n, cols, vals, mask)
    return CSR(n, rowptr, col, val, grid=(gx, gy, gz), node=node_of_row,
               name=f"fe27_{m}_s{seed}", meta={"elements_alive": int(alive.sum()), "margin": margin})


def q1_laplace(N: int, keep_zeros: bool = False):
    """Trilinear (Q1) FE Laplacian on [0,1]^3 with N nodes per axis (h = 1/(N-1)).

    Dirichlet nodes are removed, leaving (N-2)^3 unknowns in natural order.
    Assembled interior stencil: 8h/3 on the diagonal, 0 for the 6 face
    neighbours, -h/6 for the 12 edge neighbours and -h/12 for the 8 corner
    neighbours.  The load vector is b = M_h f with the consistent Q1 mass
    matrix (tensor product of the 1D stencil h/6 [1 4 1]) applied to the nodal
    values of f = cos(x + y) at all N^3 nodes (Sec. 5.1.1).  ``keep_zeros``
    keeps the exactly-zero face couplings as explicit entries.

    Returns (A, b).
    """
    g = N - 2
    h = 1.0 / (N - 1)
    shape = (g, g, g)
    offs = _offsets27_sorted(g, g)
    n = g ** 3
    k, j, i = np.meshgrid(np.arange(g), np.arange(g), np.arange(g), indexing="ij")
    lin = (i + g * (j + g * k)).ravel()
    cols = np.empty((n, 27), dtype=np.int64)
    vals = np.empty((n, 27), dtype=np.float64)
    mask = np.empty((n, 27), dtype=bool)
    for s, d in enumerate(offs):
        nz = sum(1 for v in d if v != 0)
        coef = {0: 8.0 * h / 3.0, 1: 0.0, 2: -h / 6.0, 3: -h / 12.0}[nz]
        ii, jj, kk = i + d[0], j + d[1], k + d[2]
        ok = ((ii >= 0) & (ii < g) & (jj >= 0) & (jj < g) & (kk >= 0) & (kk < g)).ravel()
        if nz == 1 and not keep_zeros:
            ok = np.zeros_like(ok)
        cols[:, s] = lin + d[0] + g * (d[1] + g * d[2])
        vals[:, s] = coef
        mask[:, s] = ok
    rowptr, col, val = _rows_to_csr(n, cols, vals, mask)
    A = CSR(n, rowptr, col, val, grid=(g, g, g), node=None, name=f"q1_laplace_{N}")
    # load vector: b_i = sum_j M_ij f_j over all nodes j (interior and boundary)
    xs = np.arange(N) * h
    Z, Y, X = np.meshgrid(xs, xs, xs, indexing="ij")
    f = np.cos(X + Y)
    w = np.array([1.0, 4.0, 1.0]) * (h / 6.0)
    bf = np.zeros((g, g, g))
    for a, wz in enumerate(w):
        for bb, wy in enumerate(w):
            for cc, wx in enumerate(w):
                bf += wz * wy * wx * f[a:a + g, bb:bb + g, cc:cc + g]
    return A, bf.ravel()


# ---------------------------------------------------------------------------
# Local matrices of substructuring (interface block split between subdomains)
# ---------------------------------------------------------------------------

@dataclass
class LocalCSR:
    """One subdomain's local matrix A_s (Sec. 4.3, Eq. (4.5)): rows and columns
    are the nodes the subdomain knows, in local numbering, and the entries come
    from the subdomain's own elements only, so that summed over subdomains
    they give the assembled matrix; on the interface A33 = sum_s A33^(s)
    (Eq. (4.6)).  ``l2g[l]`` is the global row of local node l."""

    n: int
    rowptr: np.ndarray            # int32[n+1]
    col: np.ndarray               # int32[nnz], local indices
    val: np.ndarray               # float64[nnz]
    l2g: np.ndarray               # int32[n]

    @property
    def nnz(self) -> int:
        return int(self.rowptr[-1])


def _cell_cuts(g: int, p: int):
    """Cell boxes along one axis of g unknown nodes (indices 0..g-1, Dirichlet
    ghosts at -1 and g): cell c spans nodes c and c+1, c = -1..g-1, and box t
    holds cells [cuts[t], cuts[t+1] - 1].  Neighbouring boxes share the node
    plane cuts[t], t = 1..p-1, which is floor(t g / p): the separator planes
    of the node-based substructuring."""
    if p < 1 or p > g:
        raise ValueError("need 1 <= subdomains per axis <= nodes per axis")
    return [-1] + [(t * g) // p for t in range(1, p)] + [g]


def cell_box_locals(kind: str, m, sub) -> list:
    """Local matrices of ``laplace7(m)`` (kind "laplace7") or of
    ``q1_laplace(m)`` (kind "q1", m = nodes per axis including the boundary)
    split into px*py*pz subdomains of grid cells.

    Both operators are sums of per-cell element matrices over the cells of the
    grid, Dirichlet ghost cells included:
      laplace7: 3/4 on the diagonal and -1/4 between the two ends of each of
                the cell's 12 edges (8 cells give 6, 4 cells give -1);
      q1:       the trilinear stiffness of a cube of side h = 1/(m-1): h/3 on
                the diagonal, 0 along an edge, -h/12 across a face or the body
                diagonal (the zero couplings are not stored).
    Subdomain s = sx + px (sy + py sz) assembles its own box of cells, so
    every entry is (element entry) x (number of the box's cells holding both
    nodes).  Nodes on the shared planes belong to 2, 4 or 8 subdomains.
    Rows keep their entries in ascending local column order.
    """
    if kind == "laplace7":
        gx, gy, gz = _grid_dims(m)
        offs = [(dx, dy, dz) for (dx, dy, dz) in _OFF7]
        coef = {0: 0.75, 1: -0.25}
    elif kind == "q1":
        N = int(m)
        gx = gy = gz = N - 2
        h = 1.0 / (N - 1)
        offs = [(dx, dy, dz) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)
                if sum(1 for v in (dx, dy, dz) if v) != 1]
        coef = {0: h / 3.0, 2: -h / 12.0, 3: -h / 12.0}
    else:
        raise ValueError(f"unknown kind {kind!r}")
    px, py, pz = (int(v) for v in sub)
    cuts = [_cell_cuts(g, p) for g, p in ((gx, px), (gy, py), (gz, pz))]
    dims = (gx, gy, gz)

    def axis_count(a, d, clo, chi, g):
        # cells of [clo, chi] holding node a and node a+d (d in -1, 0, 1) along one axis
        if d == 0:
            return (((a - 1 >= clo) & (a - 1 <= chi)).astype(np.int64) + ((a >= clo) & (a <= chi)))
        c = np.minimum(a, a + d)
        return ((c >= clo) & (c <= chi) & (a + d >= 0) & (a + d < g)).astype(np.int64)

    out = []
    for sz in range(pz):
        for sy in range(py):
            for sx in range(px):
                box = (sx, sy, sz)
                lo = [max(cuts[a][box[a]], 0) for a in range(3)]
                hi = [min(cuts[a][box[a] + 1], dims[a] - 1) for a in range(3)]
                ln = [hi[a] - lo[a] + 1 for a in range(3)]
                coords = [np.arange(lo[a], hi[a] + 1) for a in range(3)]
                nl = ln[0] * ln[1] * ln[2]
                cols = np.empty((nl, len(offs)), dtype=np.int64)
                vals = np.empty((nl, len(offs)), dtype=np.float64)
                mask = np.empty((nl, len(offs)), dtype=bool)
                lin = np.arange(nl).reshape(ln[2], ln[1], ln[0])
                for e, d in enumerate(offs):
                    cnt = [axis_count(coords[a], d[a], cuts[a][box[a]], cuts[a][box[a] + 1] - 1, dims[a])
                           for a in range(3)]
                    c3 = cnt[2][:, None, None] * cnt[1][None, :, None] * cnt[0][None, None, :]
                    k = coef[sum(1 for v in d if v)]
                    cols[:, e] = (lin + d[0] + ln[0] * (d[1] + ln[1] * d[2])).ravel()
                    vals[:, e] = (k * c3).ravel()
                    mask[:, e] = (c3 > 0).ravel()
                rowptr, col, val = _rows_to_csr(nl, cols, vals, mask)
                Z, Y, X = np.meshgrid(coords[2], coords[1], coords[0], indexing="ij")
                l2g = (X + gx * (Y + gy * Z)).ravel().astype(np.int32)
                out.append(LocalCSR(nl, rowptr, col, val, l2g))
    return out


# ---------------------------------------------------------------------------
# Right-hand sides, batches and the paper's small examples
# ---------------------------------------------------------------------------

def solution_and_rhs(A: CSR, seed: int, nrhs: int = 1) -> Tuple[np.ndarray, np.ndarray]:
    """x* ~ U[-1, 1] from ``seed`` and b = A x*.  Shapes (n,) or (n, nrhs)."""
    rng = np.random.default_rng(seed)
    if nrhs == 1:
        xs = rng.uniform(-1.0, 1.0, size=A.n)
    else:
        xs = rng.uniform(-1.0, 1.0, size=(A.n, nrhs))
    return xs, A.scipy() @ xs


def uniform_rhs(n: int, seed: int, nrhs: int = 1) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return rng.uniform(-1.0, 1.0, size=(n,) if nrhs == 1 else (n, nrhs))


def batch_grid_edges(nsys: int, seed: int, lo: int = 8, hi: int = 48) -> np.ndarray:
    """Grid edges m_s = round(exp(U[ln lo, ln hi])) for ``nsys`` systems."""
    rng = np.random.default_rng(seed)
    return np.rint(np.exp(rng.uniform(math.log(lo), math.log(hi), size=nsys))).astype(np.int64)


def laplace7_batch(nsys: int, seed: int, nrhs: int = 4, lo: int = 8, hi: int = 48):
    """``nsys`` independent 7-point Laplace systems with log-uniform grid edges,
    each with ``nrhs`` right-hand sides b ~ U[-1, 1] (row-major n x nrhs).

    Returns (list of CSR, list of b arrays)."""
    ms = batch_grid_edges(nsys, seed, lo, hi)
    cache = {}
    mats, rhs = [], []
    rng = np.random.default_rng(seed + 1_000_003)
    for m in ms:
        m = int(m)
        if m not in cache:
            cache[m] = laplace7(m)
        A = cache[m]
        mats.append(A)
        rhs.append(rng.uniform(-1.0, 1.0, size=(A.n, nrhs)))
    return mats, rhs


def paper_csr_example() -> np.ndarray:
    """The 5x5 matrix of the paper's CSR illustration (Sec. 4.1, matrix A)."""
    return np.array([
        [-5.0, 14.0, 0.0, 0.0, 0.0],
        [0.0, 8.0, 1.0, 0.0, 0.0],
        [2.0, 0.0, 10.0, 0.0, 0.0],
        [0.0, 4.0, 0.0, 2.0, 9.0],
        [0.0, 0.0, 15.0, 0.0, 7.0],
    ])


def paper_pattern_10x10() -> np.ndarray:
    """Boolean 10x10 non-zero pattern of the paper's three-band example
    (Sec. 4.2.2, figure of splitting a matrix into three band rows)."""
    rows = {
        1: (1, 2, 4, 6), 2: (1, 2, 3, 5), 3: (2, 3, 4, 5), 4: (1, 3, 4, 7, 10),
        5: (3, 5, 7), 6: (1, 6, 7, 9), 7: (3, 5, 6, 7, 10), 8: (2, 4, 8, 10),
        9: (6, 9), 10: (4, 7, 8, 10),
    }
    P = np.zeros((10, 10), dtype=bool)
    for r, cs in rows.items():
        for c in cs:
            P[r - 1, c - 1] = True
    return P


def dense_to_csr(Ad: np.ndarray) -> CSR:
    """Input helper: a dense matrix (tiny tests only) as 0-based CSR."""
    S = sp.csr_matrix(Ad)
    S.sort_indices()
    return CSR(Ad.shape[0], S.indptr.astype(np.int32), S.indices.astype(np.int32),
               S.data.astype(np.float64), name="dense")


def random_dominant(n: int, seed: int, density: float = 0.05, margin: float = 0.2,
                    symmetric: bool = False) -> CSR:
    """Random sparse strictly diagonally dominant matrix (tiny tests)."""
    rng = np.random.default_rng(seed)
    M = (rng.random((n, n)) < density) * rng.uniform(-1.0, 1.0, size=(n, n))
    if symmetric:
        M = np.triu(M, 1)
        M = M + M.T
    np.fill_diagonal(M, 0.0)
    d = (1.0 + margin) * np.abs(M).sum(axis=1) + 0.5
    sign = np.where(rng.random(n) < 0.5, -1.0, 1.0)
    np.fill_diagonal(M, d * sign)
    return dense_to_csr(M)


def random_irregular(n: int, seed: int, long_rows: int = 2, long_len: int = 3000, margin: float = 0.1) -> CSR:
    """Sparse strictly diagonally dominant matrix with an irregular row-length
    mix: most rows 2-8 off-diagonal entries, a quarter 9-40, a few 41-200, and
    ``long_rows`` rows of ``long_len`` entries (longer than a staged tile).
    Columns uniform over the other rows, values U[-1, 1], each row's entries
    stored in random column order."""
    rng = np.random.default_rng(seed)
    u = rng.random(n)
    lens = np.where(u < 0.70, rng.integers(2, 9, n), np.where(u < 0.95, rng.integers(9, 41, n),
                                                               rng.integers(41, 201, n)))
    for r in rng.choice(n, size=min(long_rows, n), replace=False):
        lens[r] = long_len
    lens = np.minimum(lens, n - 1)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    cols, vals = [], []
    for i in range(n):
        c = rng.choice(n - 1, size=int(lens[i]), replace=False)
        c = c + (c >= i)                          # skip the diagonal
        v = rng.uniform(-1.0, 1.0, size=c.size)
        d = (1.0 + margin) * np.abs(v).sum() + 0.1
        d = d if rng.random() < 0.5 else -d
        k = rng.integers(0, c.size + 1)           # the diagonal at a random place in the row
        cols.append(np.insert(c, k, i))
        vals.append(np.insert(v, k, d))
        rowptr[i + 1] = rowptr[i] + c.size + 1
    return CSR(n, rowptr.astype(np.int32), np.concatenate(cols).astype(np.int32), np.concatenate(vals),
               name=f"irregular_{n}_{seed}")
