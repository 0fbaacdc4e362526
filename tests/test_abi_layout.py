"""The binding's ctypes structures against the C header: every field at the
offset and of the size a C compiler gives it, and every structure of the
same total size (a field added to include/jacobi.h but not to the binding
changes the size).  Needs gcc, no GPU."""
import ctypes
import os
import shutil
import subprocess

import pytest

from conftest import ROOT
from paper_2112_02377_gb300 import jacobi as J

STRUCTS = [("jac_csr", J.jac_csr), ("jac_local", J.jac_local), ("jac_opts", J.jac_opts),
           ("jac_stats_t", J.jac_stats_t)]


def _c_layout(tmp_path):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "jacobi.h"', "int main(void) {"]
    for cname, cls in STRUCTS:
        lines.append(f'    printf("{cname} . %zu %zu\\n", sizeof({cname}), (size_t)0);')
        for fname, _ in cls._fields_:
            lines.append(f'    printf("{cname} {fname} %zu %zu\\n", offsetof({cname}, {fname}), '
                         f'sizeof((({cname}*)0)->{fname}));')
    lines += ["    return 0;", "}"]
    src = os.path.join(tmp_path, "layout.c")
    with open(src, "w") as f:
        f.write("\n".join(lines) + "\n")
    exe = os.path.join(tmp_path, "layout")
    subprocess.check_call([cc, "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), src, "-o", exe])
    out = subprocess.run([exe], capture_output=True, text=True, check=True, timeout=60).stdout
    got = {}
    for line in out.splitlines():
        s, fld, a, b = line.split()
        got[(s, fld)] = (int(a), int(b))
    return got


def test_ctypes_structures_match_the_header(tmp_path):
    got = _c_layout(str(tmp_path))
    for cname, cls in STRUCTS:
        assert ctypes.sizeof(cls) == got[(cname, ".")][0], cname
        for fname, ftype in cls._fields_:
            off, size = got[(cname, fname)]
            desc = getattr(cls, fname)
            assert (desc.offset, desc.size) == (off, size), f"{cname}.{fname}"
            assert ctypes.sizeof(ftype) == size, f"{cname}.{fname}"


def _header_prototypes():
    import re
    s = open(os.path.join(ROOT, "include", "jacobi.h")).read()
    s = re.sub(r"/\*.*?\*/", "", s, flags=re.S)
    out = {}
    for m in re.finditer(r"(?m)^([a-z_0-9 ]+\**)\s*\b(jac_[a-z_]+)\s*\(([^)]*)\)\s*;", s):
        params = [" ".join(p.split()) for p in m.group(3).split(",")]
        out[m.group(2)] = (" ".join(m.group(1).split()), params)
    return out


def _ctype_of(decl: str):
    if "*" in decl:
        return ctypes.c_void_p
    base = decl.split()[-2] if len(decl.split()) > 1 else decl
    return {"int32_t": ctypes.c_int32, "int64_t": ctypes.c_int64, "double": ctypes.c_double,
            "jac_splitting": ctypes.c_int32, "jac_status": ctypes.c_int32}[base]


def test_ctypes_signatures_match_the_header():
    protos = _header_prototypes()
    L = J.lib()
    assert sorted(protos) == sorted(J.EXPORTED)
    for name, (ret, params) in protos.items():
        f = getattr(L, name)
        want_ret = {"void": None, "jac_status": ctypes.c_int32, "const char*": ctypes.c_char_p}[ret]
        assert f.restype == want_ret, name
        want_args = [_ctype_of(p) for p in params]
        assert list(f.argtypes) == want_args, name
