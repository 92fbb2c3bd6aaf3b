"""CPU-side checks of the C-ABI library (no GPU work is launched).

The library must load, export every function include/rac_admm.h declares,
agree with the ctypes structure layouts, and reject invalid arguments
before touching the device.
"""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "rac_admm.h")


@pytest.fixture(scope="module")
def lib():
    from paper_1907_01995_gb300 import build as B
    B.build()
    from paper_1907_01995_gb300 import _lib
    return _lib.load()


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = set(re.findall(r"\b(rac_[a-z0-9_]+)\s*\(", src))
    return sorted(names)


def test_header_declares_functions():
    names = declared_functions()
    for must in ("rac_admm_setup", "rac_admm_solve", "rac_admm_batch", "rac_admm_path",
                 "rac_admm_checkpoint", "rac_admm_restore", "rac_admm_destroy"):
        assert must in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_struct_layout_matches_c(tmp_path, lib):
    """Compile a C program against the header and compare sizeof/offsetof
    with the ctypes mirrors used by the binding."""
    from paper_1907_01995_gb300 import _lib as L
    prog = tmp_path / "layout.c"
    fields = {"rac_problem": L.RacProblem, "rac_options": L.RacOptions, "rac_info": L.RacInfo}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "rac_admm.h"',
             "int main(void) {"]
    for cname, cls in fields.items():
        lines.append('printf("%s %%zu\\n", sizeof(%s));' % (cname, cname))
        for f, _ in cls._fields_:
            lines.append('printf("%s.%s %%zu\\n", offsetof(%s, %s));' % (cname, f, cname, f))
    lines.append("return 0; }")
    prog.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-I" + os.path.join(ROOT, "include"), str(prog), "-o", str(exe)])
    out = dict(line.rsplit(" ", 1) for line in subprocess.check_output([str(exe)]).decode().split("\n") if line)
    for cname, cls in fields.items():
        assert int(out[cname]) == ctypes.sizeof(cls), cname
        for f, _ in cls._fields_:
            assert int(out["%s.%s" % (cname, f)]) == getattr(cls, f).offset, (cname, f)


def test_invalid_arguments_rejected_without_gpu(lib):
    from paper_1907_01995_gb300 import _lib as L
    pr = L.RacProblem()
    o = L.RacOptions()
    assert lib.rac_options_default(ctypes.byref(o)) == 0
    h = ctypes.c_void_p()
    # no data at all
    assert lib.rac_admm_setup(ctypes.byref(pr), ctypes.byref(o), ctypes.byref(h)) == L.RAC_ERR_ARG
    # more blocks than coordinates
    import numpy as np
    A = np.zeros((4, 3), order="F")
    pr.A, pr.m, pr.n, pr.lda = A.ctypes.data, 4, 3, 4
    o.num_blocks = 4
    assert lib.rac_admm_setup(ctypes.byref(pr), ctypes.byref(o), ctypes.byref(h)) == L.RAC_ERR_ARG
    o.num_blocks = 1
    pr.lda = 2   # lda < m
    assert lib.rac_admm_setup(ctypes.byref(pr), ctypes.byref(o), ctypes.byref(h)) == L.RAC_ERR_ARG
    pr.lda = 4
    pr.phi = 2
    pr.lo, pr.hi = 1.0, 0.0   # empty box
    assert lib.rac_admm_setup(ctypes.byref(pr), ctypes.byref(o), ctypes.byref(h)) == L.RAC_ERR_ARG
    assert h.value is None
    # RP-MBADMM on the handle needs equal blocks (n = 3, p = 2 is refused);
    # unknown assembly modes
    pr.phi = 0
    o.assembly = 1
    o.num_blocks = 2
    assert lib.rac_admm_setup(ctypes.byref(pr), ctypes.byref(o), ctypes.byref(h)) == L.RAC_ERR_ARG
    o.num_blocks = 1
    o.assembly = 2
    assert lib.rac_admm_setup(ctypes.byref(pr), ctypes.byref(o), ctypes.byref(h)) == L.RAC_ERR_ARG
    xo = (ctypes.c_void_p * 1)(None)
    assert lib.rac_admm_batch(1, ctypes.byref(pr), ctypes.byref(o), xo, None) == L.RAC_ERR_ARG
    o.assembly = 0
    assert h.value is None
    assert lib.rac_assembly(0, 1, 0, 0, 1, None, None, None) == L.RAC_ERR_ARG
    # sparse data: only the residual form, and not together with a dense A
    colptr = np.array([0, 1, 2, 2], dtype=np.int64)
    rowidx = np.array([0, 3], dtype=np.int32)
    vals = np.array([1.0, 2.0])
    ps = L.RacProblem()
    ps.m, ps.n, ps.nnz = 4, 3, 2
    ps.colptr, ps.rowidx, ps.vals = colptr.ctypes.data, rowidx.ctypes.data, vals.ctypes.data
    o.form = 1   # RAC_FORM_GRAM
    assert lib.rac_admm_setup(ctypes.byref(ps), ctypes.byref(o), ctypes.byref(h)) == L.RAC_ERR_ARG
    o.form = 0
    ps.A, ps.lda = A.ctypes.data, 4
    assert lib.rac_admm_setup(ctypes.byref(ps), ctypes.byref(o), ctypes.byref(h)) == L.RAC_ERR_ARG
    assert h.value is None
    assert lib.rac_status_string(4).decode() == "block matrix not positive definite"


def test_box_qp_mode_arguments_rejected_without_gpu(lib):
    """The box kept in the block argmins needs phi = box, the Gram form, k <= 1,
    the RAC assembly, blocks of at most 128 coordinates and box_prox >= 0;
    the batch does not take it."""
    import numpy as np
    from paper_1907_01995_gb300 import _lib as L
    n = 300
    H = np.eye(n)
    pr = L.RacProblem()
    pr.m, pr.n, pr.H = n, n, H.ctypes.data
    pr.phi, pr.lo, pr.hi = 2, 0.0, 1.0
    o = L.RacOptions()
    assert lib.rac_options_default(ctypes.byref(o)) == 0
    h = ctypes.c_void_p()
    o.box_qp, o.num_blocks = 1, 2              # blocks of 150 > 128
    assert lib.rac_admm_setup(ctypes.byref(pr), ctypes.byref(o), ctypes.byref(h)) == L.RAC_ERR_ARG
    o.num_blocks = 3
    for field, bad in (("box_qp", 2), ("box_prox", -1.0), ("box_prox", float("nan")),
                       ("assembly", 1), ("form", 2)):
        old = getattr(o, field)
        setattr(o, field, bad)
        assert lib.rac_admm_setup(ctypes.byref(pr), ctypes.byref(o), ctypes.byref(h)) == L.RAC_ERR_ARG, field
        setattr(o, field, old)
    pr.phi = 1                                 # not a box
    assert lib.rac_admm_setup(ctypes.byref(pr), ctypes.byref(o), ctypes.byref(h)) == L.RAC_ERR_ARG
    pr.phi = 2
    E = np.ones((2, n))
    pr.E, pr.k, pr.d = E.ctypes.data, 2, np.zeros(2).ctypes.data   # k = 2 rows
    assert lib.rac_admm_setup(ctypes.byref(pr), ctypes.byref(o), ctypes.byref(h)) == L.RAC_ERR_ARG
    pr.k = 0
    xo = (ctypes.c_void_p * 1)(None)
    assert lib.rac_admm_batch(1, ctypes.byref(pr), ctypes.byref(o), xo, None) == L.RAC_ERR_ARG
    assert h.value is None
