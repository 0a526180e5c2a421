"""Explicit Jacobian of the CPD residual, for tests on tiny sizes only.

Built entry by entry from Lemma "partialf" (Sec. 3.4): the derivative of
f_{i1..iL} with respect to w_{i' r'}^(l') is -prod_{l≠l'} w_{il r'}^(l) when
i' = i_l', else 0.  Rows are the entries of T in column-major order (the
row order does not change J^T J or J^T f); columns follow the stacked vec
w = [vec W^(1); ...; vec W^(L)] (Sec. 3.1).
"""
from __future__ import annotations

import itertools

import numpy as np


def param_offsets(dims, R):
    offs, o = [], 0
    for d in dims:
        offs.append(o)
        o += d * R
    return offs, o


def explicit_jacobian(Ws) -> np.ndarray:
    dims = [W.shape[0] for W in Ws]
    R = Ws[0].shape[1]
    L = len(dims)
    offs, n = param_offsets(dims, R)
    N = int(np.prod(dims))
    J = np.zeros((N, n))
    # column-major enumeration of the entries
    for row, idx in enumerate(itertools.product(*[range(d) for d in reversed(dims)])):
        idx = tuple(reversed(idx))
        for lp in range(L):
            for r in range(R):
                v = 1.0
                for l in range(L):
                    if l != lp:
                        v *= Ws[l][idx[l], r]
                J[row, offs[lp] + r * dims[lp] + idx[lp]] = -v
    return J


def stack(Vs) -> np.ndarray:
    """w = [vec V^(1); ...; vec V^(L)], vec stacking columns."""
    return np.concatenate([V.ravel(order="F") for V in Vs])


def unstack(w, dims, R):
    out, o = [], 0
    for d in dims:
        out.append(w[o:o + d * R].reshape((d, R), order="F"))
        o += d * R
    return out
