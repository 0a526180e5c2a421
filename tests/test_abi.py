"""The C-ABI library loads and exports every entry point include/cpd.h
declares; option defaults are the thesis's; host-side validation rejects bad
arguments before any launch (CPU only: nothing here touches a GPU)."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def cpd():
    from paper_2110_05997_gb300 import build as b
    b.build()
    from paper_2110_05997_gb300 import cpd as m
    m.lib()
    return m


def _declared():
    names = []
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            src = open(os.path.join(ROOT, "include", f)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"^\s*(?:[A-Za-z_][A-Za-z0-9_]*[\s*]+)+(cpd_[a-z_0-9]+)\s*\(", src, re.M)
    return sorted(set(names))


def test_every_declared_symbol_is_exported(cpd):
    names = _declared()
    assert "cpd_dgn_solve" in names and "cpd_batch_solve" in names and "cpd_compress" in names
    L = cpd.lib()
    for n in names:
        assert hasattr(L, n), n
    assert sorted(cpd.EXPORTS) == names


def test_defaults_are_the_thesis_defaults(cpd):
    o = cpd.cpd_default_options()
    # Sec. 4.1.3 main parameters and Sec. 4.4 fine-tuning result
    assert o.maxiter == 200 and o.tol == 1e-6 and o.tau == 1.0
    assert o.cg_a == 0.4 and o.cg_b == 0.9
    assert o.st_mlsvd == 1 and o.compress == 1 and o.init == 0
    # the FP32 damping floor (not in the thesis) and the default wait budget
    assert o.mu_min == 1e-5 and o.timeout_cycles == 0 and o.precond == 0
    assert cpd.cpd_status_string(-1) == "invalid argument"


def test_struct_layouts_match_the_header(cpd, tmp_path):
    # sizes and field offsets of the ABI structs as the host C compiler lays them out
    import shutil
    import subprocess
    cc = shutil.which("cc") or shutil.which("gcc")
    if cc is None:
        pytest.skip("no host C compiler")
    fields = {"cpd_options": [f[0] for f in cpd.cpd_options._fields_],
              "cpd_info": [f[0] for f in cpd.cpd_info._fields_]}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "cpd.h"', 'int main(void){']
    for st, fs in fields.items():
        lines.append(f'printf("{st} size %zu\\n", sizeof({st}));')
        for f in fs:
            lines.append(f'printf("{st} {f} %zu\\n", offsetof({st}, {f}));')
    lines.append("return 0;}")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    for ln in out:
        if not ln:
            continue
        st, what, val = ln.split()
        cls = getattr(cpd, st)
        if what == "size":
            assert C.sizeof(cls) == int(val), (st, C.sizeof(cls), val)
        else:
            assert getattr(cls, what).offset == int(val), (st, what)


def test_validation_before_launch(cpd):
    L = cpd.lib()
    o = cpd.cpd_default_options()
    info = cpd.cpd_info()
    nul = C.c_void_p(0)
    dummy = C.c_void_p(0x1000)   # never dereferenced: validation fails first

    def solve(L_, dims, R, opts=o, T=dummy, W=dummy, lam=dummy, ws=dummy, wsb=1 << 20):
        return L.cpd_dgn_solve(T, 0, L_, cpd._dims(dims), R, C.byref(opts), nul, W, lam,
                               C.byref(info), nul, ws, wsb, nul)

    assert solve(5, (2, 2, 2, 2, 2), 2) == -6          # order 5 unsupported
    assert solve(2, (4, 4), 2) == -6
    assert solve(3, (4, 4, 4), 0) == -1                # R = 0
    assert solve(3, (4, 0, 4), 2) == -1                # empty mode
    assert solve(3, (2, 2, 2), 9) == -1                # R > prod dims
    assert solve(3, (4, 4, 4), 65) == -6               # R above the supported maximum
    assert solve(3, (4, 4, 4), 2, T=nul) == -1         # null tensor
    assert solve(3, (4, 4, 4), 2, ws=nul) == -1        # null workspace
    bad = cpd.cpd_default_options(maxiter=0)
    assert solve(3, (4, 4, 4), 2, opts=bad) == -1
    bad = cpd.cpd_default_options(init=2)               # given init without W0
    assert solve(3, (4, 4, 4), 2, opts=bad) == -1
    bad = cpd.cpd_default_options(block_threads=100)
    assert solve(3, (4, 4, 4), 2, opts=bad) == -1
    bad = cpd.cpd_default_options(mu_min=-1.0)
    assert solve(3, (4, 4, 4), 2, opts=bad) == -1
    bad = cpd.cpd_default_options(timeout_cycles=-5)
    assert solve(3, (4, 4, 4), 2, opts=bad) == -1
    bad = cpd.cpd_default_options(precond=2)
    assert solve(3, (4, 4, 4), 2, opts=bad) == -1
    blk = cpd.cpd_default_options(precond="block")     # R x R FP64 blocks: ranks up to 32
    assert solve(3, (40, 40, 40), 33, opts=blk) == -6
    # dGN on T itself (one CTA, 32-bit entry indices) is refused beyond 2^31 - 1024
    # entries, before anything is sized or launched
    o_unc = cpd.cpd_default_options(compress=0)
    assert solve(3, (1300, 1300, 1300), 5, opts=o_unc) == -6
    assert cpd.cpd_workspace_size((1300, 1300, 1300), 5, o_unc) == 0
    # FP64 input only for the uncompressed path
    assert L.cpd_dgn_solve(dummy, 1, 3, cpd._dims((4, 4, 4)), 2, C.byref(o), nul, dummy, dummy,
                           C.byref(info), nul, dummy, 1 << 20, nul) == -6
    # a workspace that is too small is reported, not overrun
    o2 = cpd.cpd_default_options(compress=0)
    assert solve(3, (20, 20, 20), 5, opts=o2, wsb=64) == -3
    assert cpd.cpd_workspace_size((20, 20, 20), 5, o2) > 64


def test_workspace_size_grows_with_problem(cpd):
    o = cpd.cpd_default_options()
    a = cpd.cpd_workspace_size((50, 50, 50), 5, o)
    b = cpd.cpd_workspace_size((200, 200, 200), 10, o)
    assert 0 < a < b
    assert cpd.cpd_workspace_size((4, 4, 4, 4, 4), 2, o) == 0


def test_refinement_shape_limits_are_checked_before_launch(cpd):
    """The refinement pass keeps one row of the first mode per thread (up to 4
    rows for ranks <= 16), the factor blocks of the other modes twice and
    I_1 x (33 + padded R) floats in one CTA's shared memory; shapes beyond
    that are refused up front (nothing is launched, the dummy pointers are
    never touched)."""
    L = cpd.lib()
    info = cpd.cpd_info()
    nul = C.c_void_p(0)
    dummy = C.c_void_p(0x1000)

    def solve(dims, R, refine):
        o = cpd.cpd_default_options(refine_maxiter=refine)
        return L.cpd_dgn_solve(dummy, 0, len(dims), cpd._dims(dims), R, C.byref(o), nul, dummy, dummy,
                               C.byref(info), nul, dummy, 1 << 20, nul)

    def evaluate(dims, R):
        return L.cpd_refine_eval(dummy, len(dims), cpd._dims(dims), R, dummy, dummy, dummy, nul, 0, nul)

    for dims, R in [((2000, 4, 4), 2),            # I_1 above 1024
                    ((600, 4, 4), 20),            # ranks 17..32: I_1 up to 512
                    ((300, 4, 4), 40),            # ranks 33..64: I_1 up to 256
                    ((100, 4000, 4000), 16),      # factor blocks of modes 2..3 beyond shared memory
                    ((8, 2, 2, 2), 65)]:          # rank above the maximum (refused earlier)
        assert solve(dims, R, 5) == -6, (dims, R)
        assert evaluate(dims, R) == -6, (dims, R)
