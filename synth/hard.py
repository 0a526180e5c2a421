"""Seeded generators of the hard tensors the thesis benchmarks against
(Sec. 4.3.3-4.3.6 and Sec. 4.8.1): inputs only, none of the method's
arithmetic.  Layout as in synth: column-major tensors, Iℓ×R factors.

Readings of the text, where it is silent or garbled:
  * border rank (Sec. 4.3.3): x^(ℓ), y^(ℓ) are i.i.d. N(0, I) vectors (the
    text only asks for linear independence);
  * collinear factors (Sec. 4.3.5): the fixed column q^(i') of each Q is
    column 1, so x^(1) = (1 + c) q^(1) and x^(i) = q^(1) + c q^(i);
  * double bottleneck (Sec. 4.3.6): the text writes x^(i) = q^(i') for
    i >= 3, which would repeat one column R - 2 times; its own sentence
    ("the remaining columns are equal to the columns of the QR
    decomposition") gives x^(i) = q^(i), the reading taken here;
  * noise nu (Sec. 4.3.5-4.3.6) is absolute: T + nu·N with N i.i.d. N(0,1);
  * RGH family (Sec. 4.8.1): the identity is r x r (the text's "15 x 15"
    matches only r = 15), N_i is 15 x r, the perturbation 1e-3 E/||E|| is
    added to T'/||T'||.
"""
from __future__ import annotations

import numpy as np

from . import planted_tensor, rng


def outer3(a, b, c):
    return np.einsum("i,j,k->ijk", a, b, c)


def border_rank(seed: int, dims=(20, 20, 20)):
    """The rank-3 tensor of border rank 2 (Sec. 4.3.3):
    T = x1⊗x2⊗y3 + x1⊗y2⊗x3 + y1⊗x2⊗x3.  Returns (T, x, y) with x, y the
    lists of mode vectors; T is the limit of the rank-2 sequence
    border_rank_sequence(x, y, n)."""
    g = rng(seed)
    x = [g.standard_normal(I) for I in dims]
    y = [g.standard_normal(I) for I in dims]
    T = outer3(x[0], x[1], y[2]) + outer3(x[0], y[1], x[2]) + outer3(y[0], x[1], x[2])
    return np.asfortranarray(T), x, y


def border_rank_sequence(x, y, n: float):
    """T^(n) = n (x1 + y1/n)⊗(x2 + y2/n)⊗(x3 + y3/n) - n x1⊗x2⊗x3 (rank <= 2)."""
    a = [xi + yi / n for xi, yi in zip(x, y)]
    return np.asfortranarray(n * outer3(*a) - n * outer3(*x))


def matmul_tensor(N: int):
    """M_N in R^{N^2 x N^2 x N^2} (Sec. 4.3.4): sum_{i,j,k} vec(e_ij) ⊗ vec(e_jk)
    ⊗ vec(e_ik), vec column-major (entry (i, j) of an N x N matrix at i + N j)."""
    M = np.zeros((N * N, N * N, N * N))
    for i in range(N):
        for j in range(N):
            for k in range(N):
                M[i + N * j, j + N * k, i + N * k] = 1.0
    return np.asfortranarray(M)


def strassen_rank(N: int) -> int:
    """R = ceil(N^{log2 7}), the rank the thesis approximates M_N with."""
    return int(np.ceil(N ** np.log2(7.0) - 1e-12))


def _q_factors(g, dims, R):
    Qs = []
    for I in dims:
        Q, _ = np.linalg.qr(g.standard_normal((I, R)))
        Qs.append(Q)
    return Qs


def swamp(seed: int, dims=(300, 300, 300), R: int = 15, c: float = 0.5, nu: float = 0.01,
          dtype=np.float32):
    """Collinear factors in every mode (Sec. 4.3.5): x^(i) = q^(1) + c q^(i)
    (x^(1) = (1 + c) q^(1)), q the columns of the Q of a Gaussian matrix;
    T = [[X, Y, Z]] + nu N.  Returns (T, factors, T without noise)."""
    g = rng(seed)
    Qs = _q_factors(g, dims, R)
    Ws = [np.asfortranarray(Q[:, :1] + c * Q) for Q in Qs]
    T0 = planted_tensor(Ws)
    T = T0 + nu * g.standard_normal(T0.shape)
    return np.asfortranarray(T.astype(dtype)), Ws, T0


def double_bottleneck(seed: int, dims=(300, 300, 300), R: int = 15, c: float = 0.5, nu: float = 0.01,
                      dtype=np.float32):
    """Two collinear columns per mode (Sec. 4.3.6): columns 1, 2 as in swamp(),
    the others the orthonormal q^(i); T = [[X, Y, Z]] + nu N."""
    g = rng(seed)
    Qs = _q_factors(g, dims, R)
    Ws = []
    for Q in Qs:
        W = Q.copy()
        W[:, :2] = Q[:, :1] + c * Q[:, :2]
        Ws.append(np.asfortranarray(W))
    T0 = planted_tensor(Ws)
    T = T0 + nu * g.standard_normal(T0.shape)
    return np.asfortranarray(T.astype(dtype)), Ws, T0


def rgh_cholesky(r: int, c: float):
    """Upper triangular R_c with R_c^T R_c = c 1 1^T + (1 - c) I_r."""
    A = c * np.ones((r, r)) + (1.0 - c) * np.eye(r)
    return np.linalg.cholesky(A).T


def rgh(seed: int, r: int = 15, c: float = 0.5, s: int = 2, n: int = 15, dtype=np.float32):
    """A member of the 15 x 15 x 15 family of Sec. 4.8.1: A_i = N_i R_c
    diag(10^{ks/(3r)}), k = 1..r, T' = [[A_1, A_2, A_3]],
    T = T'/||T'|| + 1e-3 E/||E||.  Returns (T, factors A_i)."""
    g = rng(seed)
    Rc = rgh_cholesky(r, c)
    D = np.diag(10.0 ** (np.arange(1, r + 1) * s / (3.0 * r)))
    As = [np.asfortranarray(g.standard_normal((n, r)) @ Rc @ D) for _ in range(3)]
    Tp = planted_tensor(As)
    E = g.standard_normal(Tp.shape)
    T = Tp / np.linalg.norm(Tp) + 1e-3 * E / np.linalg.norm(E)
    return np.asfortranarray(T.astype(dtype)), As
