"""Compression by truncated MLSVD (thesis Sec. 2.2 and Sec. 4.1.1), FP64.

* Left singular vectors of an unfolding through the eigen-decomposition of its
  Gram matrix M M^T (App. A: Lemma "svd-transpose" and the theorem after it;
  Sec. 2.2 remarks this is how the MLSVD is computed).
* Classic truncated MLSVD: Algorithm "MLSVD" (Sec. 2.2).
* Sequentially truncated MLSVD: Algorithm "ST-MLSVD" (Sec. 2.2, after
  Vannieuwenhoven et al.).
* Tolerance truncation: Algorithm "Compression" (Sec. 4.1.1): smallest
  R~_l in 1..P_l, P_l = min(I_l, R), whose discarded energy ratio
  sum_{r>R~} sigma_r^2 / sum_{r<=P} sigma_r^2 is below mlsvd_tol / L.
"""
from __future__ import annotations

import numpy as np

from .tensor import unfold, mode_product


def _fix_signs(U: np.ndarray) -> np.ndarray:
    """Singular vectors are defined up to sign; make the largest-|.| entry of
    each column positive (first such entry on ties)."""
    U = U.copy()
    for r in range(U.shape[1]):
        i = int(np.argmax(np.abs(U[:, r])))
        if U[i, r] < 0:
            U[:, r] = -U[:, r]
    return U


def gram_left_singular(M: np.ndarray, P: int | None = None):
    """Left singular vectors and singular values of M (m×n) from the
    eigenpairs of the Gram matrix M M^T (App. A): sigma_k = sqrt(|lambda_k|),
    in descending order; the first P are returned."""
    G = M @ M.T
    lam, V = np.linalg.eigh(G)
    order = np.argsort(-np.abs(lam), kind="stable")
    lam, V = lam[order], V[:, order]
    if P is not None:
        lam, V = lam[:P], V[:, :P]
    return _fix_signs(V), np.sqrt(np.abs(lam))


def truncation_rank(sigma: np.ndarray, P: int, mlsvd_tol: float, L: int) -> int:
    """Algorithm "Compression" (Sec. 4.1.1): the smallest i in 1..P with
    sum_{r>i} sigma_r^2 / sum_{r<=P} sigma_r^2 < mlsvd_tol / L.  The ratio is
    of squared singular values, as in the display preceding the algorithm."""
    s2 = np.asarray(sigma[:P], dtype=np.float64) ** 2
    total = s2.sum()
    if total <= 0.0:
        return 1
    for i in range(1, P + 1):
        rel = s2[i:].sum() / total
        if rel < mlsvd_tol / L:
            return i
    return P


def mlsvd_classic(T: np.ndarray, P=None):
    """Algorithm "MLSVD": SVD of every unfolding of T, then
    S = (U1^T, ..., UL^T)·T.  P (list) caps the number of singular vectors."""
    L = T.ndim
    Us, sigmas = [], []
    for l in range(L):
        U, s = gram_left_singular(unfold(T, l), None if P is None else P[l])
        Us.append(U)
        sigmas.append(s)
    S = T
    for l in range(L):
        S = mode_product(S, Us[l].T, l)
    return Us, sigmas, S


def mlsvd_st(T: np.ndarray, P=None, ranks_fn=None):
    """Algorithm "ST-MLSVD": for l = 1..L, SVD of the mode-l unfolding of the
    partially projected tensor, truncate, and project before the next mode.
    ``ranks_fn(l, sigma)`` chooses the kept rank of mode l (default: P[l])."""
    L = T.ndim
    S = T
    Us, sigmas = [], []
    for l in range(L):
        U, s = gram_left_singular(unfold(S, l), None if P is None else P[l])
        k = U.shape[1] if ranks_fn is None else ranks_fn(l, s)
        U = U[:, :k]
        Us.append(U)
        sigmas.append(s)
        S = mode_product(S, U.T, l)
    return Us, sigmas, S


def compress(T: np.ndarray, R: int, mlsvd_tol: float = 1e-6, st: bool = True):
    """Algorithm "Compression" (Sec. 4.1.1) on top of the classic or the
    sequentially truncated MLSVD.  Returns (Us, sigmas, S, ranks), with
    sigmas the first P_l singular values of each (sequential) unfolding."""
    L = T.ndim
    P = [min(T.shape[l], R) for l in range(L)]
    if st:
        ranks = []

        def pick(l, s):
            k = truncation_rank(s, P[l], mlsvd_tol, L)
            ranks.append(k)
            return k
        Us, sigmas, S = mlsvd_st(T, P, pick)
        return Us, sigmas, S, ranks
    Us, sigmas, S = mlsvd_classic(T, P)
    ranks = [truncation_rank(sigmas[l], P[l], mlsvd_tol, L) for l in range(L)]
    Us = [Us[l][:, :ranks[l]] for l in range(L)]
    S = S[tuple(slice(0, k) for k in ranks)]
    return Us, sigmas, np.asfortranarray(S), ranks
