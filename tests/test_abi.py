"""The C-ABI library builds, loads without a GPU, exports every entry point
declared in include/bddc.h, and rejects invalid arguments on the host before
any device work."""
import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    from paper_0911_5730_gb300 import bddc
    return bddc.load()


def _declared():
    src = open(os.path.join(ROOT, "include", "bddc.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(bddc_[a-z_0-9]+)\s*\(", src)))


def test_exports_every_declared_symbol(lib):
    names = _declared()
    assert "bddc_setup" in names and "bddc_pcg_solve" in names and "bddc_submit" in names
    for name in names:
        assert hasattr(lib, name), name


def test_binding_covers_header():
    from paper_0911_5730_gb300 import bddc
    assert set(_declared()) <= set(bddc.SYMBOLS)


def _setup(lib, nx, k, e2s, nsub, levels=2, tau=float("inf"), s2=None, n2=0, cons=1, prec=0):
    from paper_0911_5730_gb300 import bddc
    k = np.ascontiguousarray(k, np.float64)
    e2s = np.ascontiguousarray(e2s, np.int32)
    dec = bddc.Decomp(e2s.ctypes.data_as(C.POINTER(C.c_int32)), nsub,
                      None if s2 is None else s2.ctypes.data_as(C.POINTER(C.c_int32)), n2)
    opts = bddc.Opts(cons, -1, prec, 0, 0)
    h = C.c_void_p()
    code = lib.bddc_setup(C.byref(bddc.Mesh(nx, nx)), k.ctypes.data_as(C.c_void_p), C.byref(dec),
                          levels, tau, C.byref(opts), None, C.byref(h))
    return code, h


def test_invalid_arguments_rejected_on_host(lib):
    nx = 8
    e2s = np.zeros(nx * nx, np.int32)
    code, h = _setup(lib, nx, np.ones(nx * nx), e2s, 1, levels=4)
    assert code == -1 and not h.value
    assert b"levels" in lib.bddc_last_error()
    code, _ = _setup(lib, nx, -np.ones(nx * nx), e2s, 1)
    assert code == -1 and b"positive" in lib.bddc_last_error()
    code, _ = _setup(lib, nx, np.ones(nx * nx), e2s, 1, levels=3)
    assert code == -1 and b"sub1_to_sub2" in lib.bddc_last_error()
    code, _ = _setup(lib, nx, np.ones(nx * nx), e2s, 1, cons=9)
    assert code == -1
    code, _ = _setup(lib, nx, np.ones(nx * nx), e2s, 1, prec=7)
    assert code == -1
    assert lib.bddc_apply(None, None, None, 1, 1, None) == -1
    assert lib.bddc_pcg_solve(None, None, None, 1, 1, 1e-8, 10, None, None) == -1


def test_binding_struct_layouts_match_header(tmp_path):
    """The ctypes structures of the binding have the sizes and field offsets
    that a C compiler gives the header's structures (a C program built from
    include/bddc.h prints them)."""
    import shutil
    import subprocess
    from paper_0911_5730_gb300 import bddc
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    pairs = {"bddc_mesh": bddc.Mesh, "bddc_decomp": bddc.Decomp, "bddc_opts": bddc.Opts,
             "bddc_solve_info": bddc.SolveInfo, "bddc_info": bddc.Info}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "bddc.h"', "int main(void) {"]
    for cname, py in pairs.items():
        lines.append('printf("%s sizeof %%zu\\n", sizeof(%s));' % (cname, cname))
        for f, _ in py._fields_:
            lines.append('printf("%s %s %%zu\\n", offsetof(%s, %s));' % (cname, f, cname, f))
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True, capture_output=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l.strip()}
    for cname, py in pairs.items():
        assert got[(cname, "sizeof")] == C.sizeof(py), cname
        for f, _ in py._fields_:
            assert got[(cname, f)] == getattr(py, f).offset, (cname, f)
