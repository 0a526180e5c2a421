"""Pins for the oracle's tensor-algebra primitives (CPU only)."""
import itertools

import numpy as np
import pytest

import oracle as O
from conftest import read_golden


def _example_tensor():
    # frontal slices of the Sec. 2.1.1 example: t_ijk = 1 + i + 3j + 12k (0-based)
    T = np.zeros((3, 4, 2))
    for i, j, k in itertools.product(range(3), range(4), range(2)):
        T[i, j, k] = 1 + i + 3 * j + 12 * k
    return T


def _parse_blocks(lines):
    blocks, i = {}, 0
    while i < len(lines):
        name, r, c = lines[i].split()
        r, c = int(r), int(c)
        blocks[name] = np.array([[float(v) for v in lines[i + 1 + k].split()] for k in range(r)])
        assert blocks[name].shape == (r, c)
        i += 1 + r
    return blocks


def test_unfolding_worked_example():
    T = _example_tensor()
    # the frontal slices as printed
    assert T[:, :, 0].tolist() == [[1, 4, 7, 10], [2, 5, 8, 11], [3, 6, 9, 12]]
    blocks = _parse_blocks(read_golden("unfolding_3x4x2.txt"))
    for l in range(3):
        np.testing.assert_array_equal(O.unfold(T, l), blocks[f"T_({l + 1})"])
        np.testing.assert_array_equal(O.fold(O.unfold(T, l), l, T.shape), T)


def test_mode_product_worked_example():
    T = _example_tensor()
    blocks = _parse_blocks(read_golden("mode_product_example.txt"))
    S = O.mode_product(T, blocks["M"], 0)
    assert S.shape == (2, 4, 2)
    np.testing.assert_array_equal(O.unfold(S, 0), blocks["(TxM)_(1)"])
    # printed frontal slices
    assert S[:, :, 1].tolist() == [[130, 157, 184, 211], [172, 208, 244, 280]]


def test_mode_product_brute_force():
    g = np.random.default_rng(1)
    T = g.standard_normal((3, 4, 5))
    M = g.standard_normal((2, 4))
    S = O.mode_product(T, M, 1)
    for a, b, c in itertools.product(range(3), range(2), range(5)):
        assert abs(S[a, b, c] - sum(M[b, j] * T[a, j, c] for j in range(4))) < 1e-12


def test_multilinear_is_sum_over_core():
    # (M1, M2, M3)·S = sum_{ijk} s_ijk M1[:,i] ⊗ M2[:,j] ⊗ M3[:,k] (Tucker form, Sec. 2.2)
    g = np.random.default_rng(2)
    S = g.standard_normal((2, 3, 2))
    Ms = [g.standard_normal((4, 2)), g.standard_normal((3, 3)), g.standard_normal((5, 2))]
    ref = np.zeros((4, 3, 5))
    for i, j, k in itertools.product(range(2), range(3), range(2)):
        ref += S[i, j, k] * np.einsum("a,b,c->abc", Ms[0][:, i], Ms[1][:, j], Ms[2][:, k])
    np.testing.assert_allclose(O.multilinear(Ms, S), ref, rtol=0, atol=1e-12)


def test_kron_khatri_rao_definitions_and_gram_identity():
    g = np.random.default_rng(3)
    A, B = g.standard_normal((3, 4)), g.standard_normal((5, 4))
    K = O.kron(A, B)
    # B's index fastest
    assert abs(K[1 * 5 + 2, 3 * 4 + 1] - A[1, 3] * B[2, 1]) < 1e-14
    KR = O.khatri_rao(A, B)
    for r in range(4):
        for i, j in itertools.product(range(3), range(5)):
            assert abs(KR[i * 5 + j, r] - A[i, r] * B[j, r]) < 1e-14
    # App. B, Theorem "special products" item 11: (A⊙B)^T(A⊙B) = A^TA * B^TB
    np.testing.assert_allclose(KR.T @ KR, (A.T @ A) * (B.T @ B), rtol=1e-12)


@pytest.mark.parametrize("dims,R", [((3, 4, 2), 2), ((2, 3, 2, 3), 3)])
def test_cpd_tensor_brute_force(dims, R):
    g = np.random.default_rng(4)
    Ws = [g.standard_normal((d, R)) for d in dims]
    lam = g.standard_normal(R)
    T = O.cpd_tensor(Ws, lam)
    for idx in itertools.product(*[range(d) for d in dims]):
        v = sum(lam[r] * np.prod([Ws[l][idx[l], r] for l in range(len(dims))]) for r in range(R))
        assert abs(T[idx] - v) < 1e-12
    # the unfolding identity of Sec. 2.2 (Kolda): T_(l) = W_l (others ⊙, reversed)^T
    for l in range(len(dims)):
        Wl = Ws[l] * (lam[None, :] if l == 0 else 1.0)
        others = [Ws[j] * (lam[None, :] if j == 0 else 1.0) for j in range(len(dims)) if j != l]
        K = others[-1]
        for W in reversed(others[:-1]):
            K = O.khatri_rao(K, W)
        np.testing.assert_allclose(O.unfold(T, l), Wl @ K.T, atol=1e-12)
