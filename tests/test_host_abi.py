"""CPU tests of the C ABI: the library loads, exports every declared symbol,
and its host-side splitting / dependency-list logic equals the oracle's
(bit-exact integer work).  No GPU work is launched here."""
import os
import re

import numpy as np
import pytest

from conftest import ROOT, golden_path
from oracle import oracle as O
from paper_2112_02377_gb300 import jacobi as J
from paper_2112_02377_gb300 import workloads as W


def _header_functions():
    src = open(os.path.join(ROOT, "include", "jacobi.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(jac_[a-z_]+)\s*\(", src)))


def test_library_loads_and_exports_every_declared_symbol():
    L = J.lib()
    declared = _header_functions()
    assert len(declared) >= 16
    for name in declared:
        assert hasattr(L, name), name
    assert sorted(J.EXPORTED) == declared


def _matrices():
    yield "lap7_12", W.laplace7(12), None
    yield "lap7_box", W.laplace7((9, 7, 11)), None
    yield "diff7", W.diffusion7((10, 8, 6), seed=3), None
    F = W.fe27_deleted(9, seed=1)
    yield "fe27", F, F.node


@pytest.mark.parametrize("name,A,node", list(_matrices()))
def test_band_splittings_match_oracle(name, A, node):
    for P in (1, 2, 3, 7, 64):
        perm, parts = J.jac_partition_plan(A, J.JAC_BANDROW, P)
        assert np.array_equal(perm, np.arange(A.n))
        assert np.array_equal(parts, O.band_row_parts(A.n, P))
        perm, parts = J.jac_partition_plan(A, J.JAC_BANDROW_NNZ, P)
        assert np.array_equal(parts, O.band_nnz_parts(A.rowptr, P))


@pytest.mark.parametrize("name,A,node", list(_matrices()))
def test_substructuring_matches_oracle(name, A, node):
    for sub in [(1, 1, 1), (2, 2, 2), (3, 2, 1), (2, 1, 3)]:
        o = J.opts(grid=A.grid, subdomains=sub)
        perm, parts = J.jac_partition_plan(A, J.JAC_SUBSTRUCT, 0, o, node_of_row=node)
        p2, pp2 = O.substructure(A.grid, sub, A.n, node=node)
        assert np.array_equal(perm, p2)
        assert np.array_equal(parts, pp2)


def test_substructuring_160_cube_interface_size():
    A = W.laplace7(40)
    o = J.opts(grid=(40, 40, 40), subdomains=(4, 4, 4))
    perm, parts = J.jac_partition_plan(A, J.JAC_SUBSTRUCT, 0, o)
    assert len(parts) == 66
    assert parts[-1] - parts[-2] == 40 ** 3 - 37 ** 3


@pytest.mark.parametrize("name,A,node", list(_matrices()))
def test_dependency_lists_match_oracle(name, A, node):
    for s, P in [(J.JAC_BANDROW, 4), (J.JAC_BANDROW_NNZ, 5)]:
        rptr, rfrom, recv = J.jac_dependency_lists(A, s, P)
        parts = O.band_row_parts(A.n, P) if s == J.JAC_BANDROW else O.band_nnz_parts(A.rowptr, P)
        rcv, _ = O.dependency_lists(A.rowptr, A.col, parts)
        hp, h = O.halo_of(rcv)
        assert np.array_equal(rptr[: P + 1], hp)
        assert np.array_equal(recv, h)
        owner = O.owner_of_rows(parts, np.arange(A.n), A.n)
        assert np.array_equal(rfrom, owner[recv])
    o = J.opts(grid=A.grid, subdomains=(2, 2, 2))
    rptr, rfrom, recv = J.jac_dependency_lists(A, J.JAC_SUBSTRUCT, 0, o, node_of_row=node)
    perm, parts = O.substructure(A.grid, (2, 2, 2), A.n, node=node)
    rcv, _ = O.dependency_lists(A.rowptr, A.col, parts, perm)
    hp, h = O.halo_of(rcv)
    assert np.array_equal(rptr[: len(hp)], hp)
    assert np.array_equal(recv, h)
    # interiors receive only from the interface (Eq. (4.4) block structure)
    S = len(parts) - 2
    for p in range(S):
        assert np.all(rfrom[rptr[p]:rptr[p + 1]] == S)


def test_dependency_lists_reproduce_paper_example():
    pat = W.paper_pattern_10x10()
    A = W.dense_to_csr(pat.astype(float) + 10 * np.eye(10))
    rptr, rfrom, recv = J.jac_dependency_lists(A, J.JAC_BANDROW, 3)
    got = {}
    for p in range(3):
        for q, j in zip(rfrom[rptr[p]:rptr[p + 1]], recv[rptr[p]:rptr[p + 1]]):
            got.setdefault((p + 1, int(q) + 1), []).append(int(j) + 1)
    want = {}
    for line in open(golden_path("dependency_10x10_3bands.txt")):
        line = line.split("#")[0].strip()
        if line.startswith("recv"):
            head, nodes = line.split(":")
            _, a, _, b = head.split()
            want[(int(a), int(b))] = [int(v) for v in nodes.split()]
    assert got == want


def test_one_based_input_is_accepted():
    A = W.laplace7(6)
    A1 = W.CSR(A.n, A.rowptr + 1, A.col + 1, A.val)
    csr, keep = J.make_csr(A1.rowptr, A1.col, A1.val, A.n, index_base=1)
    import ctypes
    perm = np.empty(A.n, dtype=np.int64)
    part = np.empty(4, dtype=np.int64)
    cnt = ctypes.c_int64()
    st = J.lib().jac_partition_plan(ctypes.byref(csr), J.JAC_BANDROW_NNZ, 3, ctypes.byref(J.opts()),
                                    ctypes.c_void_p(perm.ctypes.data), ctypes.c_void_p(part.ctypes.data),
                                    ctypes.byref(cnt))
    assert st == J.JAC_OK
    assert np.array_equal(part, O.band_nnz_parts(A.rowptr, 3))


@pytest.mark.parametrize("mutate,msg", [
    ("col_range", "column index out of range"),
    ("rowptr_dec", "rowptr decreases"),
    ("nparts0", "nparts"),
    ("nparts_big", "nparts"),
    ("sub_nogrid", "grid"),
    ("sub_coupled", "coupled"),
    ("sub_toomany", "subdomains"),
    ("nonfinite", "non-finite"),
])
def test_invalid_inputs_are_rejected(mutate, msg):
    A = W.laplace7(6)
    rp, col, val = A.rowptr.copy(), A.col.copy(), A.val.copy()
    s, P, o = J.JAC_BANDROW, 3, J.opts()
    if mutate == "col_range":
        col[5] = A.n
    elif mutate == "rowptr_dec":
        rp[10] = rp[12]
    elif mutate == "nparts0":
        P = 0
    elif mutate == "nparts_big":
        P = A.n + 1
    elif mutate == "sub_nogrid":
        s = J.JAC_SUBSTRUCT
    elif mutate == "sub_coupled":
        s, o = J.JAC_SUBSTRUCT, J.opts(grid=(3, 12, 6), subdomains=(2, 2, 2))
    elif mutate == "sub_toomany":
        s, o = J.JAC_SUBSTRUCT, J.opts(grid=(6, 6, 6), subdomains=(7, 1, 1))
    elif mutate == "nonfinite":
        val[3] = np.nan
    B = W.CSR(A.n, rp, col, val)
    with pytest.raises(J.JacobiError) as ei:
        J.jac_partition_plan(B, s, P, o)
    assert ei.value.status == J.JAC_EINVAL
    assert msg in str(ei.value)


def test_setup_without_a_gpu_fails_loudly():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    A = W.laplace7(4)
    with pytest.raises(J.JacobiError) as ei:
        J.jac_setup(A, np.ones(A.n), J.JAC_BANDROW, 2)
    assert ei.value.status == J.JAC_ECUDA


def test_autotune_rejects_a_fixed_geometry_before_touching_the_gpu():
    A = W.laplace7(4)
    b = np.ones(A.n)
    for kw in (dict(variant=2), dict(tile_rows=256), dict(ctas_per_sm=3)):
        with pytest.raises(J.JacobiError) as e:
            J.jac_setup(A, b, J.JAC_BANDROW, 1, J.opts(autotune=1, **kw))
        assert "autotune" in str(e.value)
    with pytest.raises(J.JacobiError) as e:
        J.jac_setup_batched([A], [b], J.opts(autotune=1, tile_rows=96))
    assert "autotune" in str(e.value)


@pytest.mark.parametrize("case,msg", [
    ("nrhs3", "nrhs must be 1, 2 or 4"),
    ("no_systems", "nsys"),
    ("stages5", "stages"),
    ("sync7", "sync"),
])
def test_batched_inputs_are_checked_before_any_device_call(case, msg):
    A = W.laplace7(4)
    As, bs, o = [A], [np.ones(A.n)], J.opts()
    if case == "nrhs3":
        o = J.opts(nrhs=3)
    elif case == "no_systems":
        As, bs = [], []
    elif case == "stages5":
        o = J.opts(stages=5)
    elif case == "sync7":
        o = J.opts(sync=7)
    with pytest.raises(J.JacobiError) as ei:
        J.jac_setup_batched(As, bs, o)
    assert ei.value.status == J.JAC_EINVAL and msg in str(ei.value)


def test_empty_system_is_rejected():
    E = W.CSR(0, np.zeros(1, dtype=np.int32), np.zeros(0, dtype=np.int32), np.zeros(0))
    with pytest.raises(J.JacobiError) as ei:
        J.jac_partition_plan(E, J.JAC_BANDROW, 1, J.opts())
    assert ei.value.status == J.JAC_EINVAL and "empty" in str(ei.value)


@pytest.mark.parametrize("field,value,msg", [
    ("lanes_per_row", 3, "lanes_per_row"),
    ("stages", 5, "stages"),
    ("sync", 7, "sync"),
    ("tile_rows", 100, "tile_rows"),
    ("ctas_per_sm", 4, "ctas_per_sm"),
    ("inner_sweeps", 1, "inner_sweeps"),
    ("norm", 1, "norm"),
])
def test_option_values_are_checked_before_any_device_call(field, value, msg):
    A = W.laplace7(4)
    with pytest.raises(J.JacobiError) as ei:
        J.jac_setup(A, np.ones(A.n), J.JAC_BANDROW, 2, J.opts(**{field: value}))
    assert ei.value.status == J.JAC_EINVAL and msg in str(ei.value)


def test_irregular_workload_shape_and_scipy_copy_keeps_stored_order():
    """The irregular input has unsorted rows, a diagonal at a random place and
    strict row dominance; handing it to scipy (which sorts in place) must not
    reorder the caller's entries, since the entry order fixes every row sum."""
    A = W.random_irregular(3000, 3)
    lens = np.diff(A.rowptr)
    assert lens.max() == min(3001, A.n) and (lens >= 3).all()
    col0, val0 = A.col.copy(), A.val.copy()
    unsorted = sum(np.any(np.diff(A.col[A.rowptr[i]:A.rowptr[i + 1]]) < 0) for i in range(A.n))
    assert unsorted > A.n // 2
    _ = abs(A.scipy()) @ np.ones(A.n)
    assert np.array_equal(A.col, col0) and np.array_equal(A.val, val0)
    D = A.scipy()
    diag = np.abs(D.diagonal())
    off = np.asarray(abs(D).sum(axis=1)).ravel() - diag
    assert (diag > off).all()


# ------------------------------------------------ split interface (jac_setup_local) ----

def _star_locals(nsub):
    """nsub subdomains, each holding node 0 and one node of its own (node 0
    is on the interface of all of them)."""
    locs = []
    for s in range(nsub):
        locs.append(W.LocalCSR(2, np.array([0, 2, 4], np.int32), np.array([0, 1, 0, 1], np.int32),
                               np.array([4.0, -1.0, -1.0, 4.0]), np.array([0, s + 1], np.int32)))
    return locs, nsub + 1


def _edit(L, **kw):
    d = dict(n=L.n, rowptr=L.rowptr, col=L.col, val=L.val, l2g=L.l2g)
    d.update(kw)
    return W.LocalCSR(**d)


@pytest.mark.parametrize("case,status,msg", [
    ("uncovered", "EINVAL", "belongs to no subdomain"),
    ("repeated_l2g", "EINVAL", "listed twice"),
    ("l2g_range", "EINVAL", "out of range"),
    ("col_range", "EINVAL", "column index out of range"),
    ("two_diag", "EINVAL", "two diagonal entries"),
    ("zero_diag", "ESINGULAR", "assembled diagonal"),
    ("crowded", "EINVAL", "held by 9 subdomains"),
    ("mixed", "EINVAL", "FP64"),
    ("async", "EINVAL", "grid sync"),
])
def test_split_interface_inputs_are_checked_before_any_device_call(case, status, msg):
    locs = W.cell_box_locals("laplace7", 4, (2, 1, 1))
    n, o = 64, J.opts()
    if case == "uncovered":
        locs = locs[:1]
    elif case == "repeated_l2g":
        g = locs[0].l2g.copy()
        g[1] = g[0]
        locs[0] = _edit(locs[0], l2g=g)
    elif case == "l2g_range":
        g = locs[1].l2g.copy()
        g[-1] = 64
        locs[1] = _edit(locs[1], l2g=g)
    elif case == "col_range":
        c = locs[0].col.copy()
        c[3] = locs[0].n
        locs[0] = _edit(locs[0], col=c)
    elif case == "two_diag":
        L = locs[0]
        c = L.col.copy()
        k = int(L.rowptr[5])
        c[k] = 5 if c[k] != 5 else c[k]
        c[k + 1] = 5
        locs[0] = _edit(L, col=c)
    elif case == "zero_diag":
        locs = [_edit(L, val=np.where(L.col == np.repeat(np.arange(L.n), np.diff(L.rowptr)), 0.0, L.val))
                for L in locs]
    elif case == "crowded":
        locs, n = _star_locals(9)
        o = J.opts(lanes_per_row=4)
    elif case == "mixed":
        o = J.opts(precision=J.JAC_MIXED)
    elif case == "async":
        o = J.opts(sync=J.JAC_SYNC_ASYNC)
    with pytest.raises(J.JacobiError) as ei:
        J.jac_setup_local(n, locs, np.ones(n), o)
    assert ei.value.status == getattr(J, "JAC_" + status) and msg in str(ei.value), str(ei.value)


def test_split_interface_setup_without_a_gpu_fails_loudly():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    locs = W.cell_box_locals("laplace7", 6, (2, 2, 1))
    with pytest.raises(J.JacobiError) as ei:
        J.jac_setup_local(216, locs, np.ones(216))
    assert ei.value.status == J.JAC_ECUDA


def test_noalloc_entry_point_checks_arguments_and_reports_a_missing_device():
    """jac_sweep_noalloc rejects bad sizes before any device call and, with no
    GPU, returns JAC_ECUDA with a message (it never throws or crashes)."""
    import ctypes
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present: host pointers would reach the kernels")
    L = J.lib()
    A = W.laplace7(4)
    rp, cl, vl = A.rowptr.astype(np.int32), A.col.astype(np.int32), A.val.astype(np.float64)
    b, x0, out = np.ones(A.n), np.zeros(A.n), np.zeros(A.n)
    P = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    rel = ctypes.c_double()
    st = L.jac_sweep_noalloc(0, P(rp), P(cl), P(vl), P(b), P(x0), P(out), 1, ctypes.byref(rel), None)
    assert st == J.JAC_EINVAL and b"n must be" in L.jac_last_error(None)
    st = L.jac_sweep_noalloc(A.n, P(rp), P(cl), P(vl), P(b), P(x0), P(out), 1, ctypes.byref(rel), None)
    assert st == J.JAC_ECUDA and L.jac_last_error(None).startswith(b"jac_sweep_noalloc: ")


def test_local_stop_options_are_checked_before_any_device_call():
    """JAC_STOP_LOCAL needs FP64, the infinity norm, grid-synchronised sweeps
    and the persistent kernel with 1, 2 or 4 lanes; batched and split
    contexts keep the global test.  All rejected on the host."""
    A = W.laplace7(6)
    b = np.ones(A.n)
    bad = [dict(norm=J.JAC_NORM_REL2), dict(norm=J.JAC_NORM_INF, precision=J.JAC_MIXED),
           dict(norm=J.JAC_NORM_INF, sync=J.JAC_SYNC_NEIGHBOUR), dict(norm=J.JAC_NORM_INF, variant=1),
           dict(norm=J.JAC_NORM_INF, variant=3), dict(norm=J.JAC_NORM_INF, tile_rows=224),
           dict(norm=J.JAC_NORM_INF, lanes_per_row=8)]
    for kw in bad:
        with pytest.raises(J.JacobiError) as ei:
            J.jac_setup(A, b, J.JAC_BANDROW, 2, J.opts(stop=J.JAC_STOP_LOCAL, **kw))
        assert ei.value.status == J.JAC_EINVAL and "JAC_STOP_LOCAL" in str(ei.value), kw
    with pytest.raises(J.JacobiError) as ei:
        J.jac_setup(A, b, J.JAC_BANDROW, 2, J.opts(stop=2))
    assert ei.value.status == J.JAC_EINVAL
    with pytest.raises(J.JacobiError) as ei:
        J.jac_setup_batched([A], [b], J.opts(stop=J.JAC_STOP_LOCAL, norm=J.JAC_NORM_INF))
    assert ei.value.status == J.JAC_EINVAL
    with pytest.raises(J.JacobiError) as ei:
        J.jac_setup_local(A.n, W.cell_box_locals("laplace7", 6, (2, 1, 1)), b,
                          J.opts(stop=J.JAC_STOP_LOCAL, norm=J.JAC_NORM_INF))
    assert ei.value.status == J.JAC_EINVAL
