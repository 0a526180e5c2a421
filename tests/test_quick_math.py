"""The solver's scalar division and square root (quick_div, quick_sqrt in
csrc/common.cuh: an FP32 estimate refined by one step of Newton's method in
FP64) stay within 2^-44 relative error of the correctly rounded FP64 results
over the operand range the solver feeds them (quotients and roots of error
norms, gains and step sizes: magnitudes 1e-30 .. 1e30).  The functions are
compiled for the host by the system C++ compiler from the same header."""
import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2110_05997_gb300", "csrc")


def _nvcc():
    for p in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if p and os.path.exists(p):
            return p
    return None


def test_quick_div_and_sqrt_accuracy(tmp_path):
    nvcc = _nvcc()
    if nvcc is None:
        pytest.skip("needs nvcc")
    g = np.random.default_rng(5)
    n = 20000
    a = g.uniform(-1, 1, n) * 10.0 ** g.uniform(-30, 30, n)
    b = g.uniform(0.1, 1, n) * 10.0 ** g.uniform(-30, 30, n) * g.choice([-1, 1], n)
    x = np.abs(a)
    # the documented validity: operands and results within the FP32 normal range
    keep = (np.abs(a / b) < 1e37) & (np.abs(a / b) > 1e-37)
    a, b = a[keep], b[keep]
    inp = tmp_path / "in.txt"
    with open(inp, "w") as fh:
        for u, v, w in zip(a, b, x[keep]):
            fh.write(f"{u.hex()} {v.hex()} {w.hex()}\n")
    src = tmp_path / "q.cu"
    src.write_text('#include <cstdio>\n#include <cstdlib>\n#include "common.cuh"\n'
                   "int main(int c, char** v){ FILE* f = fopen(v[1], \"r\"); char s1[64], s2[64], s3[64];\n"
                   "while (fscanf(f, \"%63s %63s %63s\", s1, s2, s3) == 3) {\n"
                   "double a = strtod(s1, 0), b = strtod(s2, 0), x = strtod(s3, 0);\n"
                   "printf(\"%a %a\\n\", cpdk::quick_div(a, b), cpdk::quick_sqrt(x)); }\n"
                   "return 0; }\n")
    exe = tmp_path / "q"
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-std=c++17", "-Xcompiler",
                    "-ffp-contract=off", "-I", CSRC, str(src), "-o", str(exe)], check=True, capture_output=True)
    out = subprocess.run([str(exe), str(inp)], capture_output=True, text=True, check=True).stdout.split()
    q = np.array([float.fromhex(t) for t in out[0::2]])
    s = np.array([float.fromhex(t) for t in out[1::2]])
    rq = np.abs(q - a / b) / np.abs(a / b)
    rs = np.abs(s - np.sqrt(x[keep])) / np.sqrt(x[keep])
    assert rq.max() <= 2.0 ** -44, rq.max()
    assert rs.max() <= 2.0 ** -44, rs.max()
