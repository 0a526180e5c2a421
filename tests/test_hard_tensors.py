"""The hard-tensor generators (synth/hard.py) against what the thesis fixes
about each family: the border-rank tensor is the derivative of a rank-one
curve and the limit of rank-2 tensors (Sec. 4.3.3), M_N contracts two
matrices into their product (Sec. 4.3.4), the collinear and double-bottleneck
factors have the Gram matrices their construction implies (Sec. 4.3.5-4.3.6),
and the RGH factors carry the Cholesky factor of c 11^T + (1-c) I and the
geometric column scaling (Sec. 4.8.1)."""
import numpy as np
import pytest

from synth import hard


def test_border_rank_is_the_derivative_of_a_rank_one_curve():
    T, x, y = hard.border_rank(11, (7, 6, 5))
    curve = lambda t: hard.outer3(*[xi + t * yi for xi, yi in zip(x, y)])
    h = 1e-2
    central = (curve(h) - curve(-h)) / (2 * h)
    # the curve is cubic in t: the central difference is exact up to h^2 y1⊗y2⊗y3
    exact = T + h * h * hard.outer3(*y)
    assert np.allclose(central, exact, rtol=0, atol=1e-12 * np.abs(exact).max())


def test_border_rank_is_a_limit_of_rank_two_tensors():
    T, x, y = hard.border_rank(12, (8, 8, 8))
    d = [np.linalg.norm(hard.border_rank_sequence(x, y, n) - T) for n in (100.0, 200.0, 400.0)]
    # T^(n) - T = (x1⊗y2⊗y3 + y1⊗x2⊗y3 + y1⊗y2⊗x3)/n + y1⊗y2⊗y3/n^2
    assert 1.9 < d[0] / d[1] < 2.1 and 1.9 < d[1] / d[2] < 2.1
    lead = np.linalg.norm(hard.outer3(x[0], y[1], y[2]) + hard.outer3(y[0], x[1], y[2]) + hard.outer3(y[0], y[1], x[2]))
    assert abs(d[2] * 400.0 - lead) <= 0.01 * lead


@pytest.mark.parametrize("N", [2, 3, 4])
def test_matmul_tensor_contracts_to_the_matrix_product(N):
    M = hard.matmul_tensor(N)
    g = np.random.default_rng(N)
    A, B = g.standard_normal((N, N)), g.standard_normal((N, N))
    got = np.einsum("abc,a,b->c", M, A.ravel(order="F"), B.ravel(order="F"))
    assert np.allclose(got, (A @ B).ravel(order="F"), atol=1e-12)
    assert M.sum() == N ** 3 and set(np.unique(M)) <= {0.0, 1.0}


def test_strassen_rank():
    assert [hard.strassen_rank(n) for n in (2, 3, 4, 5)] == [7, 22, 49, 92]


@pytest.mark.parametrize("c", [0.1, 0.5, 0.9])
def test_swamp_factor_grams(c):
    T, Ws, T0 = hard.swamp(3, (20, 18, 16), 6, c, nu=0.01, dtype=np.float64)
    R = 6
    e1 = np.zeros(R); e1[0] = 1.0
    expect = np.ones((R, R)) + c * (e1[:, None] + e1[None, :]) + c * c * np.eye(R)
    for W in Ws:
        assert np.allclose(W.T @ W, expect, atol=1e-12)
    n = np.linalg.norm(T - T0) / np.sqrt(T.size)
    assert abs(n - 0.01) < 0.001                     # absolute noise of standard deviation nu


@pytest.mark.parametrize("c", [0.1, 0.5])
def test_double_bottleneck_factor_grams(c):
    T, Ws, T0 = hard.double_bottleneck(4, (20, 18, 16), 6, c, nu=0.01, dtype=np.float64)
    expect = np.eye(6)
    expect[:2, :2] = [[(1 + c) ** 2, 1 + c], [1 + c, 1 + c * c]]
    for W in Ws:
        assert np.allclose(W.T @ W, expect, atol=1e-12)


@pytest.mark.parametrize("r,c", [(15, 0.0), (20, 0.25), (30, 0.75)])
def test_rgh_cholesky_and_scaling(r, c):
    Rc = hard.rgh_cholesky(r, c)
    assert np.allclose(np.triu(Rc), Rc)
    assert np.allclose(Rc.T @ Rc, c * np.ones((r, r)) + (1 - c) * np.eye(r), atol=1e-12)
    T, As = hard.rgh(5, r, c, 3, dtype=np.float64)
    assert T.shape == (15, 15, 15) and all(A.shape == (15, r) for A in As)
    assert abs(np.linalg.norm(T) - 1.0) <= 1.1e-3
    # A_i diag(10^{-ks/(3r)}) R_c^{-1} is the Gaussian N_i: its columns have no scaling trend
    D = np.diag(10.0 ** (-np.arange(1, r + 1) * 3 / (3.0 * r)))
    Ng = As[0] @ D @ np.linalg.inv(Rc)
    norms = np.linalg.norm(Ng, axis=0)
    assert abs(np.polyfit(np.arange(r), np.log10(norms), 1)[0]) < 0.05
