"""Tensor algebra primitives (thesis Ch. 1-2 and App. B), FP64 numpy.

Conventions fixed by the thesis and used everywhere:
  * unfolding T_(l): rows indexed by i_l, columns ordered with i_1 fastest
    (skipping l) -- Algorithm "Unfolding" (Sec. 2.1.1) and its 3×4×2 example;
  * mode-l product S = T ×_l M: S_(l) = M · T_(l) (Sec. 2.1 definition and
    its example with M = [[1,3,5],[2,4,6]]);
  * multilinear multiplication (M1,...,ML)·T = T ×_1 M1 ... ×_L ML;
  * Kronecker product A ⊗ B with B's index fastest, Khatri-Rao product
    A ⊙ B = column-wise Kronecker (App. B, Theorem "special products");
  * a CPD [[W1,...,WL]] = sum_r w_r^(1) ⊗ ... ⊗ w_r^(L) (Sec. 3.1, eq. (compute_cpd)).
"""
from __future__ import annotations

import numpy as np


def unfold(T: np.ndarray, l: int) -> np.ndarray:
    """T_(l) in R^{I_l × prod_{j≠l} I_j}, columns with i_1 fastest (Algorithm Unfolding)."""
    I = T.shape[l]
    return np.moveaxis(np.asarray(T), l, 0).reshape(I, -1, order="F")


def fold(M: np.ndarray, l: int, dims) -> np.ndarray:
    """Inverse of ``unfold`` for a tensor of shape ``dims``."""
    dims = list(dims)
    moved = [dims[l]] + dims[:l] + dims[l + 1:]
    return np.asfortranarray(np.moveaxis(M.reshape(moved, order="F"), 0, l))


def mode_product(T: np.ndarray, M: np.ndarray, l: int) -> np.ndarray:
    """T ×_l M with M of shape (I_l', I_l): (T ×_l M)_(l) = M · T_(l)."""
    dims = list(T.shape)
    dims[l] = M.shape[0]
    return fold(M @ unfold(T, l), l, dims)


def multilinear(Ms, T: np.ndarray) -> np.ndarray:
    """(M1, ..., ML) · T = T ×_1 M1 ×_2 M2 ... ×_L ML."""
    S = T
    for l, M in enumerate(Ms):
        S = mode_product(S, M, l)
    return S


def kron(A: np.ndarray, B: np.ndarray) -> np.ndarray:
    """Kronecker product, B's index fastest (App. B)."""
    return np.kron(A, B)


def khatri_rao(A: np.ndarray, B: np.ndarray) -> np.ndarray:
    """A ⊙ B: column r is kron(a_r, b_r) (App. B)."""
    R = A.shape[1]
    assert B.shape[1] == R
    return np.stack([np.kron(A[:, r], B[:, r]) for r in range(R)], axis=1)


def kr_others(Ws, l: int) -> np.ndarray:
    """W^(L) ⊙ ... ⊙ W^(l+1) ⊙ W^(l-1) ⊙ ... ⊙ W^(1): rows follow the column
    order of T_(l) (i_1 fastest), as in the gradient theorem of Sec. 4.1.3."""
    others = [Ws[j] for j in range(len(Ws)) if j != l]
    K = others[-1]
    for W in reversed(others[:-1]):
        K = khatri_rao(K, W)
    return K


def cpd_tensor(Ws, lam=None) -> np.ndarray:
    """[[W1, ..., WL]] (optionally with weights lambda_r) as a dense tensor,
    through the unfolding identity T_(1) = W1 · (W^(L) ⊙ ... ⊙ W^(2))^T."""
    dims = [W.shape[0] for W in Ws]
    W1 = Ws[0] if lam is None else Ws[0] * np.asarray(lam)[None, :]
    if len(Ws) == 1:
        return W1.sum(axis=1)
    return fold(W1 @ kr_others(Ws, 0).T, 0, dims)
