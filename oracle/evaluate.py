"""Scoring of CPDs in FP64: explicit-residual fit and permutation/scale
alignment.  A CPD is unique only up to permutation and scaling of its
rank-one terms (Sec. 1.4 on essential uniqueness), so factors are compared
after alignment; results of both the CUDA path and the oracle are scored by
the same functions here."""
from __future__ import annotations

import numpy as np
from scipy.optimize import linear_sum_assignment

from .tensor import cpd_tensor


def fit(T: np.ndarray, Ws, lam=None) -> float:
    """||T - [[lambda; W]]|| / ||T|| from the explicit residual (FP64)."""
    T = np.asarray(T, dtype=np.float64)
    Ws = [np.asarray(W, dtype=np.float64) for W in Ws]
    E = T - cpd_tensor(Ws, None if lam is None else np.asarray(lam, dtype=np.float64))
    return float(np.linalg.norm(E) / np.linalg.norm(T))


def _unit(Ws, lam):
    nr = [np.linalg.norm(W, axis=0) for W in Ws]
    lam = np.ones(Ws[0].shape[1]) if lam is None else np.asarray(lam, np.float64).copy()
    for n in nr:
        lam = lam * n
    return [W / np.where(n > 0, n, 1.0)[None, :] for W, n in zip(Ws, nr)], lam


def align(Wa, lam_a, Wb, lam_b):
    """Match the terms of CPD a to those of CPD b maximising
    prod_l |<a_r^(l), b_s^(l)>| (Hungarian assignment).  Returns
    (perm, signs) with a-term perm[s] matched to b-term s, signs[l][s] = ±1."""
    Ua, la = _unit(Wa, lam_a)
    Ub, lb = _unit(Wb, lam_b)
    R = Ua[0].shape[1]
    C = np.ones((R, R))
    for A, B in zip(Ua, Ub):
        C = C * np.abs(A.T @ B)
    rows, cols = linear_sum_assignment(-C)
    perm = np.empty(R, dtype=int)
    perm[cols] = rows
    signs = [np.sign(np.sum(A[:, perm] * B, axis=0)) for A, B in zip(Ua, Ub)]
    return perm, signs


def compare_cpd(Wa, lam_a, Wb, lam_b):
    """Relative differences of two CPDs after alignment: per mode
    max_r ||a_r s - b_r|| for unit columns, and max_r |lambda_a - lambda_b|/lambda_b
    (the sign of a term may move between modes, so lambdas carry the product
    of the per-mode signs)."""
    Ua, la = _unit(Wa, lam_a)
    Ub, lb = _unit(Wb, lam_b)
    perm, signs = align(Wa, lam_a, Wb, lam_b)
    mode_err = []
    total_sign = np.ones(Ua[0].shape[1])
    for A, B, s in zip(Ua, Ub, signs):
        s = np.where(s == 0, 1.0, s)
        total_sign = total_sign * s
        mode_err.append(float(np.max(np.linalg.norm(A[:, perm] * s[None, :] - B, axis=0))))
    lam_err = float(np.max(np.abs(la[perm] * total_sign - lb) / np.maximum(np.abs(lb), 1e-300)))
    return dict(mode_err=mode_err, lam_err=lam_err, perm=perm)
