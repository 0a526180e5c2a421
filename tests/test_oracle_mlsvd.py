"""Pins for the oracle's compression (CPU only): the warming-up worked
example (Sec. 4.2, Table 4.5), MLSVD theorems of Sec. 2.2 as invariants, and
the truncation rule of Algorithm "Compression" (Sec. 4.1.1)."""
import itertools

import numpy as np
import pytest

import oracle as O
import synth
from conftest import read_golden


def _warm_core():
    T = synth.warming_up_tensor()
    Us, sig, S = O.mlsvd_classic(T)
    return T, Us, sig, S


def test_gram_route_matches_svd():
    # App. A: singular values of M are sqrt of the eigenvalues of M M^T and the
    # left singular vectors are its eigenvectors (checked against LAPACK's SVD)
    g = np.random.default_rng(5)
    M = g.standard_normal((6, 40)) * np.array([9, 5, 3, 2, 1, 0.5])[:, None]
    U, s = O.gram_left_singular(M)
    U2, s2, _ = np.linalg.svd(M, full_matrices=False)
    np.testing.assert_allclose(s, s2, rtol=1e-12)
    np.testing.assert_allclose(np.abs(U.T @ U2), np.eye(6), atol=1e-10)
    np.testing.assert_allclose(U.T @ U, np.eye(6), atol=1e-12)


def test_warming_up_table_4_5():
    T, Us, sig, S = _warm_core()
    St = S[:3, :3, :3]
    nS = np.linalg.norm(St)
    rows = read_golden("warming_up_table45.txt")
    assert len(rows) == 27
    for ln in rows:
        i, j, k, v = ln.split()
        sub = St[:int(i), :int(j), :int(k)]
        err = np.sqrt(max(nS ** 2 - np.linalg.norm(sub) ** 2, 0.0)) / nS
        assert abs(err - float(v)) <= 0.6e-8, (i, j, k, err, v)


def test_warming_up_rank_and_core():
    T, Us, sig, S = _warm_core()
    # multilinear rank (3,3,3): the truncated core keeps the whole norm (printed 3.85e-14)
    St = S[:3, :3, :3]
    trunc = np.sqrt(max(np.linalg.norm(S) ** 2 - np.linalg.norm(St) ** 2, 0.0)) / np.linalg.norm(S)
    assert trunc < 1e-10
    for s in sig:
        assert s[3] / s[0] < 1e-6
    lines = read_golden("warming_up_core.txt")
    slices, k = [], 0
    while lines[k].startswith("slice"):
        slices.append([[float(v) for v in lines[k + 1 + r].split()] for r in range(3)])
        k += 4
    for kk, sl in enumerate(slices):
        for i in range(3):
            for j in range(3):
                printed = sl[i][j]
                txt = f"{abs(printed):.10g}"
                # one unit in the last printed digit
                decimals = len(txt.split(".")[1]) if "." in txt else 0
                assert abs(abs(St[i, j, kk]) - abs(printed)) <= 10.0 ** -decimals + 1e-12, \
                    (i, j, kk, St[i, j, kk], printed)


def test_warming_up_mlsvd_energy_init():
    T, Us, sig, S = _warm_core()
    St = S[:3, :3, :3]
    W0 = O.init_mlsvd_energy(St, 3)
    picked = set()
    for r in range(3):
        picked.add(tuple(int(np.flatnonzero(W[:, r])[0]) + 1 for W in W0))
    assert picked == {(1, 1, 1), (2, 1, 2), (1, 2, 2)}
    err = O.fit(T, O.uncompress([U[:, :3] for U in Us], W0))
    # the thesis truncates printed values (e.g. |s_222| = 0.1659 printed 0.16)
    assert 0.0153 <= err < 0.0154


@pytest.mark.parametrize("dims", [(5, 6, 7), (4, 3, 5, 2)])
def test_mlsvd_theorems(dims):
    g = np.random.default_rng(6)
    T = g.standard_normal(dims)
    Us, sig, S = O.mlsvd_classic(T)
    L = len(dims)
    # item 1: T = (U1, ..., UL)·S with orthogonal U
    np.testing.assert_allclose(O.multilinear(Us, S), T, atol=1e-10)
    for U in Us:
        np.testing.assert_allclose(U.T @ U, np.eye(U.shape[0]), atol=1e-12)
    for l in range(L):
        Sl = O.unfold(S, l)
        G = Sl @ Sl.T
        # all-orthogonality and ||S_{i_l=k}|| = sigma_k, descending
        np.testing.assert_allclose(G - np.diag(np.diag(G)), 0, atol=1e-9)
        np.testing.assert_allclose(np.sqrt(np.diag(G)), sig[l], rtol=1e-10)
        assert np.all(np.diff(sig[l]) <= 1e-12)
        # ||T||^2 = sum sigma^2
        assert abs(np.sum(sig[l] ** 2) - np.linalg.norm(T) ** 2) < 1e-9 * np.linalg.norm(T) ** 2
    # single-mode truncation error = discarded sigma^2 (Thm "SVD-truncation" on the unfolding)
    k = 2
    Tk = O.multilinear([Us[0][:, :k] @ Us[0][:, :k].T] + [np.eye(d) for d in dims[1:]], T)
    assert abs(np.linalg.norm(T - Tk) ** 2 - np.sum(sig[0][k:] ** 2)) < 1e-9
    # multi-mode truncation bound (Thm "energy-mlsvd")
    ks = [2] * L
    St = S[tuple(slice(0, kk) for kk in ks)]
    Tt = O.multilinear([U[:, :kk] for U, kk in zip(Us, ks)], St)
    bound = sum(np.sum(s[kk:] ** 2) for s, kk in zip(sig, ks))
    assert np.linalg.norm(T - Tt) ** 2 <= bound + 1e-9


def test_st_mlsvd_exact_low_rank_and_error_bound():
    # a tensor of exact multilinear rank (2,3,2): ST and classic both reproduce it
    g = np.random.default_rng(7)
    core = g.standard_normal((2, 3, 2))
    Qs = [np.linalg.qr(g.standard_normal((d, r)))[0] for d, r in [(6, 2), (5, 3), (7, 2)]]
    T = O.multilinear(Qs, core)
    Us, sig, S, ranks = O.compress(T, 3, 1e-10, st=True)
    assert ranks == [2, 3, 2]
    np.testing.assert_allclose(O.multilinear(Us, S), T, atol=1e-10)
    Usc, sigc, Sc, ranksc = O.compress(T, 3, 1e-10, st=False)
    assert ranksc == [2, 3, 2]
    np.testing.assert_allclose(O.multilinear(Usc, Sc), T, atol=1e-10)
    # noisy tensor: ST error within the sum of discarded energies (Vannieuwenhoven et al.)
    Tn = T + 0.01 * g.standard_normal(T.shape)
    Us, sig, S = O.mlsvd_st(Tn, [2, 3, 2])
    err2 = np.linalg.norm(Tn - O.multilinear(Us, S)) ** 2
    full = O.mlsvd_st(Tn)
    bound = sum(np.sum(full[1][l][k:] ** 2) for l, k in enumerate([2, 3, 2]))
    assert err2 <= bound * (1 + 1e-9) + 1e-12


def test_truncation_rank_rule():
    # sum_{r>i} s^2 / sum_{r<=P} s^2 < tol / L, smallest such i
    s = np.array([10.0, 1.0, 0.1, 0.001])
    # ratios: i=1: (1+0.01+1e-6)/101.010001 ≈ 0.0100; i=2: 1e-4/...; i=3: 1e-8
    assert O.truncation_rank(s, 4, 3 * 0.02, 3) == 1
    assert O.truncation_rank(s, 4, 3 * 0.005, 3) == 2
    assert O.truncation_rank(s, 4, 3 * 1e-6, 3) == 3
    assert O.truncation_rank(s, 4, 3 * 1e-12, 3) == 4
    # only the first P values count: with P = 2 the ratio at i = 1 is 1/101
    assert O.truncation_rank(s, 2, 3 * 0.00991, 3) == 1
    assert O.truncation_rank(s, 2, 3 * 0.0098, 3) == 2
    # a zero spectrum keeps one vector
    assert O.truncation_rank(np.zeros(3), 3, 1e-6, 3) == 1


def test_compress_pythagoras():
    # orthonormal U: ||T - U·[[W]]||^2 = ||T||^2 - ||S||^2 + ||S - [[W]]||^2
    T, _ = synth.planted(11, (8, 7, 6), 3, 0.0, 0.05)
    Us, sig, S, ranks = O.compress(T, 3)
    g = np.random.default_rng(8)
    W = [g.standard_normal((k, 3)) for k in ranks]
    lhs = np.linalg.norm(T - O.multilinear(Us, O.cpd_tensor(W))) ** 2
    rhs = np.linalg.norm(T) ** 2 - np.linalg.norm(S) ** 2 + np.linalg.norm(S - O.cpd_tensor(W)) ** 2
    assert abs(lhs - rhs) < 1e-9 * np.linalg.norm(T) ** 2
