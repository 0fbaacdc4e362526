"""Python binding of the C ABI in ``include/jacobi.h`` (argument marshalling only).

Every function here has the name of the C entry point it calls and does
nothing but convert arguments (numpy arrays, torch tensors on the CPU or on
the GPU) into pointers and sizes, call the library, and turn error codes into
:class:`JacobiError`.  All arithmetic runs in the CUDA library
``libjacobi_gb300.so``; if it cannot be loaded the calls raise.
"""
from __future__ import annotations

import ctypes
import os
import threading
from dataclasses import dataclass
from typing import Any, Optional, Sequence, Tuple

import numpy as np

from . import _build

JAC_OK, JAC_EINVAL, JAC_ENOMEM, JAC_ECUDA, JAC_ESINGULAR, JAC_ENOTCONV, JAC_ETIMEOUT, JAC_ENUMERIC = range(8)
JAC_BANDROW, JAC_BANDROW_NNZ, JAC_SUBSTRUCT = 0, 1, 2
JAC_MEM_HOST, JAC_MEM_DEVICE = 0, 1
JAC_FP64, JAC_MIXED = 0, 1
JAC_NORM_REL2, JAC_NORM_INF = 2, 0
JAC_SYNC_GRID, JAC_SYNC_NEIGHBOUR, JAC_SYNC_ASYNC = 0, 1, 2
JAC_STOP_GLOBAL, JAC_STOP_LOCAL = 0, 1

SPLITTINGS = {"bandrow": JAC_BANDROW, "bandrow_nnz": JAC_BANDROW_NNZ, "substruct": JAC_SUBSTRUCT}
_STATUS_NAMES = ["JAC_OK", "JAC_EINVAL", "JAC_ENOMEM", "JAC_ECUDA", "JAC_ESINGULAR", "JAC_ENOTCONV",
                 "JAC_ETIMEOUT", "JAC_ENUMERIC"]

# Symbols declared in include/jacobi.h (checked by the CPU test suite).
EXPORTED = ["jac_opts_default", "jac_setup", "jac_setup_batched", "jac_setup_local", "jac_set_x", "jac_set_b", "jac_sweep",
            "jac_solve", "jac_get_x", "jac_get_history", "jac_get_batch_results", "jac_adjoint_grad",
            "jac_stats", "jac_partition_plan", "jac_dependency_lists", "jac_last_error", "jac_free",
            "jac_get_trace", "jac_sweep_noalloc"]


class JacobiError(RuntimeError):
    def __init__(self, status: int, message: str):
        self.status = status
        name = _STATUS_NAMES[status] if 0 <= status < len(_STATUS_NAMES) else str(status)
        super().__init__(f"{name}: {message}")


class jac_csr(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("nnz", ctypes.c_int64), ("rowptr", ctypes.c_void_p),
                ("col", ctypes.c_void_p), ("val", ctypes.c_void_p), ("index_base", ctypes.c_int32),
                ("memory", ctypes.c_int32)]


class jac_local(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("nnz", ctypes.c_int64), ("rowptr", ctypes.c_void_p),
                ("col", ctypes.c_void_p), ("val", ctypes.c_void_p), ("l2g", ctypes.c_void_p)]


class jac_opts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int32), ("norm", ctypes.c_int32), ("sweeps_per_graph", ctypes.c_int32),
                ("inner_sweeps", ctypes.c_int32), ("grid", ctypes.c_int32 * 3), ("subdomains", ctypes.c_int32 * 3),
                ("node_of_row", ctypes.c_void_p), ("nrhs", ctypes.c_int32), ("transpose", ctypes.c_int32),
                ("variant", ctypes.c_int32), ("tile_rows", ctypes.c_int32), ("ctas_per_sm", ctypes.c_int32),
                ("lanes_per_row", ctypes.c_int32), ("stages", ctypes.c_int32), ("sync", ctypes.c_int32),
                ("debug", ctypes.c_int32), ("autotune", ctypes.c_int32),
                ("history", ctypes.c_int32),
                ("stream", ctypes.c_void_p), ("timeout_cycles", ctypes.c_uint64),
                ("fault_skip_cta", ctypes.c_int32), ("device", ctypes.c_int32), ("stop", ctypes.c_int32)]


class jac_stats_t(ctypes.Structure):
    _fields_ = [(f, ctypes.c_int64) for f in ("n", "nnz", "nparts", "interface_rows", "ntiles", "ctas",
                                                "halo_entries", "max_row", "k", "sweeps_total",
                                                "outer_iterations", "halo_fallback_tiles",
                                                "halo_window_elems")] + \
               [(f, ctypes.c_double) for f in ("last_relres", "last_res2", "last_resinf", "last_ms",
                                                 "bytes_per_sweep_fp64", "bytes_per_sweep_fp32")] + \
               [(f, ctypes.c_int32) for f in ("variant", "precision", "splitting", "nrhs", "tile_rows",
                                                "ctas_per_sm", "lanes_per_row", "sync", "stages", "stop",
                                                "stop_part")] + \
               [("stop_local", ctypes.c_double)]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_}


_lock = threading.Lock()
_lib = None


def library_path() -> str:
    return _build.LIB


def lib(build_if_needed: bool = True):
    """Load libjacobi_gb300.so (compiling it in-tree first if it is missing or
    stale and nvcc is available).  Raises if the CUDA library cannot be loaded."""
    global _lib
    with _lock:
        if _lib is None:
            if build_if_needed:
                try:
                    _build.build()
                except Exception as e:  # no nvcc: fall through to loading what exists
                    if not os.path.exists(_build.LIB):
                        raise RuntimeError(f"CUDA library libjacobi_gb300.so is not built and cannot be built: {e}")
            if not os.path.exists(_build.LIB):
                raise RuntimeError("CUDA library libjacobi_gb300.so is missing")
            L = ctypes.CDLL(_build.LIB)
            P, I32, I64, D = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
            sig = {
                "jac_opts_default": (None, [P]),
                "jac_setup": (I32, [P, P, I32, I32, P, P]),
                "jac_setup_batched": (I32, [I32, P, P, P, P]),
                "jac_setup_local": (I32, [I64, I32, P, P, P, P]),
                "jac_set_x": (I32, [P, P, I32]),
                "jac_set_b": (I32, [P, P, I32]),
                "jac_sweep": (I32, [P, I32, P]),
                "jac_solve": (I32, [P, D, I64, P, P]),
                "jac_get_x": (I32, [P, P, I32]),
                "jac_get_history": (I32, [P, P, I64, P]),
                "jac_get_batch_results": (I32, [P, P, P]),
                "jac_adjoint_grad": (I32, [P, P, P, P, I32]),
                "jac_stats": (I32, [P, P]),
                "jac_get_trace": (I32, [P, P, P, I64, P]),
                "jac_sweep_noalloc": (I32, [I64, P, P, P, P, P, P, I32, P, P]),
                "jac_partition_plan": (I32, [P, I32, I32, P, P, P, P]),
                "jac_dependency_lists": (I32, [P, I32, I32, P, P, P, P, P]),
                "jac_last_error": (ctypes.c_char_p, [P]),
                "jac_free": (None, [P]),
            }
            for name, (res, args) in sig.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


# ----------------------------------------------------------- marshalling --

def _is_torch(a) -> bool:
    return type(a).__module__.startswith("torch")


def _buf(a, dtype, name: str, writable: bool = False):
    """(pointer, memory, keepalive) of a numpy array or torch tensor."""
    if a is None:
        return None, JAC_MEM_HOST, None
    if _is_torch(a):
        import torch
        tdt = {np.float64: torch.float64, np.int32: torch.int32, np.int64: torch.int64}[dtype]
        if a.dtype != tdt or not a.is_contiguous():
            if writable:
                raise ValueError(f"{name} must be a contiguous {tdt} tensor")
            a = a.to(tdt).contiguous()
        mem = JAC_MEM_DEVICE if a.is_cuda else JAC_MEM_HOST
        return ctypes.c_void_p(a.data_ptr()), mem, a
    arr = np.asarray(a)
    if arr.dtype != dtype or not arr.flags.c_contiguous:
        if writable:
            raise ValueError(f"{name} must be a C-contiguous {np.dtype(dtype)} array")
        arr = np.ascontiguousarray(arr, dtype=dtype)
    return ctypes.c_void_p(arr.ctypes.data), JAC_MEM_HOST, arr


def _check(st: int, ctx=None):
    if st != JAC_OK:
        msg = lib().jac_last_error(ctx).decode()
        raise JacobiError(st, msg)


def make_csr(rowptr, col, val, n: Optional[int] = None, index_base: int = 0):
    """jac_csr view of CSR arrays (numpy or torch, host or device).  Returns
    (struct, keepalive)."""
    rp, m1, k1 = _buf(rowptr, np.int32, "rowptr")
    cl, m2, k2 = _buf(col, np.int32, "col")
    vl, m3, k3 = _buf(val, np.float64, "val")
    if len({m1, m2, m3}) != 1:
        raise ValueError("rowptr, col and val must live in the same memory")
    nn = (len(rowptr) - 1) if n is None else n
    s = jac_csr(n=nn, nnz=int(len(val)), rowptr=rp, col=cl, val=vl, index_base=index_base, memory=m1)
    return s, (k1, k2, k3)


def opts(**kw) -> jac_opts:
    """jac_opts with library defaults, then the given fields."""
    o = jac_opts()
    lib().jac_opts_default(ctypes.byref(o))
    for k, v in kw.items():
        if k in ("grid", "subdomains"):
            getattr(o, k)[:] = [int(t) for t in v]
        elif k == "stream":
            o.stream = ctypes.c_void_p(int(v) if v else 0)
        elif k == "node_of_row":
            raise ValueError("pass node_of_row through jac_setup(node_of_row=...)")
        else:
            setattr(o, k, v)
    return o


# ------------------------------------------------------- entry points ----

def jac_setup(A, b=None, splitting: int = JAC_BANDROW, nparts: int = 1, o: Optional[jac_opts] = None,
              node_of_row=None, index_base: int = 0) -> ctypes.c_void_p:
    """A: object with n, rowptr, col, val (e.g. workloads.CSR) or a tuple
    (rowptr, col, val).  Returns the context handle."""
    if isinstance(A, tuple):
        csr, keep = make_csr(*A, index_base=index_base)
    else:
        csr, keep = make_csr(A.rowptr, A.col, A.val, A.n, index_base=index_base)
    bp, bm, bkeep = _buf(b, np.float64, "b")
    if b is not None and bm != csr.memory:
        raise ValueError("b must live in the same memory as A")
    o = o if o is not None else opts()
    nkeep = None
    if node_of_row is not None:
        nkeep = np.ascontiguousarray(node_of_row, dtype=np.int64)
        o.node_of_row = ctypes.c_void_p(nkeep.ctypes.data)
    ctx = ctypes.c_void_p()
    st = lib().jac_setup(ctypes.byref(csr), bp, int(splitting), int(nparts), ctypes.byref(o), ctypes.byref(ctx))
    o.node_of_row = None
    _check(st, None)
    return ctx


def jac_setup_local(n: int, locals_, b=None, o: Optional[jac_opts] = None) -> ctypes.c_void_p:
    """Substructuring with the interface block split between subdomains:
    ``locals_[s]`` has n, rowptr, col (local indices), val and l2g (e.g.
    workloads.LocalCSR), host arrays; b: n doubles (host) or None."""
    nsub = len(locals_)
    arr = (jac_local * max(nsub, 1))()
    keep = []
    for i, L in enumerate(locals_):
        rp = np.ascontiguousarray(L.rowptr, dtype=np.int32)
        cl = np.ascontiguousarray(L.col, dtype=np.int32)
        vl = np.ascontiguousarray(L.val, dtype=np.float64)
        lg = np.ascontiguousarray(L.l2g, dtype=np.int32)
        keep.append((rp, cl, vl, lg))
        arr[i] = jac_local(n=int(L.n), nnz=int(vl.size), rowptr=rp.ctypes.data, col=cl.ctypes.data,
                           val=vl.ctypes.data, l2g=lg.ctypes.data)
    bp, bm, bkeep = _buf(b, np.float64, "b")
    if b is not None and bm != JAC_MEM_HOST:
        raise ValueError("b must be host memory")
    o = o if o is not None else opts()
    ctx = ctypes.c_void_p()
    st = lib().jac_setup_local(int(n), int(nsub), arr, bp, ctypes.byref(o), ctypes.byref(ctx))
    _check(st, None)
    return ctx


def jac_setup_batched(As, bs, o: Optional[jac_opts] = None) -> ctypes.c_void_p:
    """nsys systems solved together; bs[s] is n_s x nrhs (row-major) or None."""
    nsys = len(As)
    arr = (jac_csr * nsys)()
    bp = (ctypes.c_void_p * nsys)()
    keep = []
    for i, A in enumerate(As):
        s, k = make_csr(A.rowptr, A.col, A.val, A.n)
        arr[i] = s
        keep.append(k)
    for i, b in enumerate(bs):
        p, m, k = _buf(b, np.float64, "b")
        bp[i] = p
        keep.append(k)
    o = o if o is not None else opts()
    ctx = ctypes.c_void_p()
    st = lib().jac_setup_batched(nsys, arr, bp, ctypes.byref(o), ctypes.byref(ctx))
    _check(st, None)
    return ctx


def jac_set_x(ctx, x=None):
    p, m, keep = _buf(x, np.float64, "x")
    _check(lib().jac_set_x(ctx, p, m), ctx)


def jac_set_b(ctx, b=None):
    p, m, keep = _buf(b, np.float64, "b")
    _check(lib().jac_set_b(ctx, p, m), ctx)


def jac_sweep(ctx, k: int) -> float:
    rel = ctypes.c_double()
    _check(lib().jac_sweep(ctx, int(k), ctypes.byref(rel)), ctx)
    return rel.value


def jac_solve(ctx, tol: float, maxit: int, raise_on_notconv: bool = False) -> Tuple[int, float, int]:
    """Returns (k, relres, status); raises on every status but OK / ENOTCONV."""
    k = ctypes.c_int64()
    rel = ctypes.c_double()
    st = lib().jac_solve(ctx, float(tol), int(maxit), ctypes.byref(k), ctypes.byref(rel))
    if st not in (JAC_OK, JAC_ENOTCONV) or (raise_on_notconv and st == JAC_ENOTCONV):
        _check(st, ctx)
    return int(k.value), float(rel.value), int(st)


def jac_get_x(ctx, out=None, n: Optional[int] = None):
    """Copy x^k into `out` (numpy or torch, host or device) or a new numpy array."""
    if out is None:
        if n is None:
            st = jac_stats(ctx)
            n = st["n"] * max(1, st["nrhs"])
        out = np.empty(n)
    p, m, keep = _buf(out, np.float64, "out", writable=True)
    _check(lib().jac_get_x(ctx, p, m), ctx)
    return out


def jac_get_history(ctx, max_entries: int = 1 << 30) -> np.ndarray:
    cnt = ctypes.c_int64()
    _check(lib().jac_get_history(ctx, None, int(max_entries), ctypes.byref(cnt)), ctx)
    out = np.empty(min(cnt.value, max_entries))
    _check(lib().jac_get_history(ctx, ctypes.c_void_p(out.ctypes.data), out.size, ctypes.byref(cnt)), ctx)
    return out[: cnt.value]


def jac_get_batch_results(ctx, nentries: int):
    sw = np.empty(nentries, dtype=np.int64)
    rel = np.empty(nentries)
    _check(lib().jac_get_batch_results(ctx, ctypes.c_void_p(sw.ctypes.data), ctypes.c_void_p(rel.ctypes.data)), ctx)
    return sw, rel


def jac_adjoint_grad(ctx, lam, x, dA):
    lp, lm, k1 = _buf(lam, np.float64, "lambda")
    xp, xm, k2 = _buf(x, np.float64, "x")
    gp, gm, k3 = _buf(dA, np.float64, "dA", writable=True)
    if len({lm, xm, gm}) != 1:
        raise ValueError("lambda, x and dA must live in the same memory")
    _check(lib().jac_adjoint_grad(ctx, lp, xp, gp, lm), ctx)
    return dA


def jac_get_trace(ctx):
    """Per-CTA (compute_ms, wait_ms) arrays of the last sweep/solve call."""
    n = ctypes.c_int64()
    _check(lib().jac_get_trace(ctx, None, None, 0, ctypes.byref(n)), ctx)
    comp = np.zeros(n.value)
    wait = np.zeros(n.value)
    if n.value:
        _check(lib().jac_get_trace(ctx, ctypes.c_void_p(comp.ctypes.data), ctypes.c_void_p(wait.ctypes.data),
                                   n.value, ctypes.byref(n)), ctx)
    return comp, wait


def jac_stats(ctx) -> dict:
    s = jac_stats_t()
    _check(lib().jac_stats(ctx, ctypes.byref(s)), ctx)
    return s.as_dict()


def jac_partition_plan(A, splitting: int, nparts: int, o: Optional[jac_opts] = None, node_of_row=None):
    """Host-only: (perm, part_ptr) of the splitting."""
    csr, keep = make_csr(A.rowptr, A.col, A.val, A.n)
    o = o if o is not None else opts()
    nkeep = None
    if node_of_row is not None:
        nkeep = np.ascontiguousarray(node_of_row, dtype=np.int64)
        o.node_of_row = ctypes.c_void_p(nkeep.ctypes.data)
    perm = np.empty(A.n, dtype=np.int64)
    cap = (o.subdomains[0] * o.subdomains[1] * o.subdomains[2] + 2) if splitting == JAC_SUBSTRUCT else nparts + 1
    part = np.empty(max(cap, 2), dtype=np.int64)
    np_out = ctypes.c_int64()
    st = lib().jac_partition_plan(ctypes.byref(csr), int(splitting), int(nparts), ctypes.byref(o),
                                  ctypes.c_void_p(perm.ctypes.data), ctypes.c_void_p(part.ctypes.data),
                                  ctypes.byref(np_out))
    o.node_of_row = None
    _check(st, None)
    return perm, part[: np_out.value + 1].copy()


def jac_dependency_lists(A, splitting: int, nparts: int, o: Optional[jac_opts] = None, node_of_row=None):
    """Host-only: receive lists (recv_ptr, recv_from, recv) of the splitting."""
    csr, keep = make_csr(A.rowptr, A.col, A.val, A.n)
    o = o if o is not None else opts()
    nkeep = None
    if node_of_row is not None:
        nkeep = np.ascontiguousarray(node_of_row, dtype=np.int64)
        o.node_of_row = ctypes.c_void_p(nkeep.ctypes.data)
    cap = (o.subdomains[0] * o.subdomains[1] * o.subdomains[2] + 2) if splitting == JAC_SUBSTRUCT else nparts + 1
    rptr = np.zeros(max(cap, 2), dtype=np.int64)
    tot = ctypes.c_int64()
    L = lib()
    _check(L.jac_dependency_lists(ctypes.byref(csr), int(splitting), int(nparts), ctypes.byref(o),
                                  ctypes.c_void_p(rptr.ctypes.data), None, None, ctypes.byref(tot)), None)
    rfrom = np.empty(max(tot.value, 1), dtype=np.int32)
    recv = np.empty(max(tot.value, 1), dtype=np.int64)
    _check(L.jac_dependency_lists(ctypes.byref(csr), int(splitting), int(nparts), ctypes.byref(o),
                                  ctypes.c_void_p(rptr.ctypes.data), ctypes.c_void_p(rfrom.ctypes.data),
                                  ctypes.c_void_p(recv.ctypes.data), ctypes.byref(tot)), None)
    o.node_of_row = None
    return rptr, rfrom[: tot.value], recv[: tot.value]


def jac_sweep_noalloc(rowptr, col, val, b, x_in, x_out, k: int, stream=None) -> float:
    """k sweeps without any allocation inside the library (device tensors in,
    x^k written to x_out).  Returns the relres of the last pre-update iterate
    (NaN when k == 0)."""
    ptrs = []
    for a, dt, nm in ((rowptr, np.int32, "rowptr"), (col, np.int32, "col"), (val, np.float64, "val"),
                      (b, np.float64, "b"), (x_in, np.float64, "x_in")):
        p, m, keep = _buf(a, dt, nm)
        if m != JAC_MEM_DEVICE:
            raise ValueError(f"{nm} must be in device memory")
        ptrs.append((p, keep))
    po, mo, ko = _buf(x_out, np.float64, "x_out", writable=True)
    if mo != JAC_MEM_DEVICE:
        raise ValueError("x_out must be in device memory")
    rel = ctypes.c_double(float("nan"))
    n = len(rowptr) - 1
    st = lib().jac_sweep_noalloc(n, ptrs[0][0], ptrs[1][0], ptrs[2][0], ptrs[3][0], ptrs[4][0], po, int(k),
                                 ctypes.byref(rel), ctypes.c_void_p(int(stream) if stream else 0))
    _check(st, None)
    return rel.value


def jac_last_error(ctx=None) -> str:
    return lib().jac_last_error(ctx).decode()


def jac_free(ctx):
    if ctx:
        lib().jac_free(ctx)


# ------------------------------------------------------- convenience -----

class Solver:
    """Context-managed handle around one jac_ctx."""

    def __init__(self, A, b=None, splitting="bandrow", nparts: int = 1, node_of_row=None, **kw):
        s = SPLITTINGS[splitting] if isinstance(splitting, str) else int(splitting)
        if s == JAC_SUBSTRUCT and "grid" not in kw and getattr(A, "grid", None) is not None:
            kw["grid"] = A.grid
        if node_of_row is None and getattr(A, "node", None) is not None and s == JAC_SUBSTRUCT:
            node_of_row = A.node
        self.n = A.n if not isinstance(A, tuple) else len(A[0]) - 1
        self.ctx = jac_setup(A, b, s, nparts, opts(**kw), node_of_row=node_of_row)

    def sweep(self, k: int) -> float:
        return jac_sweep(self.ctx, k)

    def solve(self, tol: float, maxit: int):
        return jac_solve(self.ctx, tol, maxit)

    def x(self, out=None):
        return jac_get_x(self.ctx, out, self.n)

    def set_x(self, x=None):
        jac_set_x(self.ctx, x)

    def set_b(self, b=None):
        jac_set_b(self.ctx, b)

    def history(self) -> np.ndarray:
        return jac_get_history(self.ctx)

    def stats(self) -> dict:
        return jac_stats(self.ctx)

    def close(self):
        if self.ctx:
            jac_free(self.ctx)
            self.ctx = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
