"""Pins for the oracle's damping update, gain ratio, regulariser and stopping
conditions (CPU only), against the rules as Sec. 4.1.3 and Sec. 4.8 print them.

Every expected value below is worked out by hand from the printed rule; the
arithmetic is in the comment beside each case.  The histories are built so
that a one-token slip in the oracle (a window edge moved by one, a missing
absolute value, a swapped order, the window constant rounded down, a norm
not squared, a squared norm where the thesis has a plain one) changes the
outcome of at least one case.
"""
import math

import numpy as np
import pytest

import oracle as O
from oracle.jacobian import explicit_jacobian

T4 = 1e-4

# (history errs[0..k], k, step, ||grad||_inf, ||S||, tol, maxiter) -> first condition
# that holds (0: none).  errs[j] is the relative error after iteration j.
STOP_CASES = [
    # -- conditions 1-4 (tol 0.01, maxiter 10) --------------------------------
    ("nothing holds", ([0.5, 0.3], 1, 1.0, 1.0, 1.0, 0.01, 10), 0),
    ("1: 0.009 < 0.01", ([0.5, 0.009], 1, 1.0, 1.0, 1.0, 0.01, 10), 1),
    ("1 is strict: 0.01 is not < 0.01", ([0.5, 0.01], 1, 1.0, 1.0, 1.0, 0.01, 10), 0),
    ("2: step 0.009 < 0.01", ([0.5, 0.3], 1, 0.009, 1.0, 1.0, 0.01, 10), 2),
    ("3: |0.305 - 0.3| < 0.01", ([0.9, 0.305, 0.3], 2, 1.0, 1.0, 1.0, 0.01, 10), 3),
    ("3 compares k-1 with k, not k-2: |0.9 - 0.3|", ([0.305, 0.9, 0.3], 2, 1.0, 1.0, 1.0, 0.01, 10), 0),
    ("4: ||grad||_inf 0.009 < 0.01", ([0.5, 0.3], 1, 1.0, 0.009, 1.0, 0.01, 10), 4),
    ("1 before 2 and 4", ([0.5, 0.005], 1, 0.005, 0.005, 1.0, 0.01, 10), 1),
    ("2 before 3 and 4", ([0.305, 0.3], 1, 0.005, 0.005, 1.0, 0.01, 10), 2),
    ("3 before 4", ([0.305, 0.3], 1, 1.0, 0.005, 1.0, 0.01, 10), 3),
    # -- condition 7: e > max(1, ||S||^2) / (1e-16 + tol) ---------------------
    ("7: ||S|| = 10 -> bound 100/0.01 = 1e4 < 2e4", ([1.0, 20000.0], 1, 1.0, 1.0, 10.0, 0.01, 10), 7),
    ("7 squares ||S||: 5000 < 1e4 (not 10/0.01 = 1000)", ([1.0, 5000.0], 1, 1.0, 1.0, 10.0, 0.01, 10), 0),
    ("7: ||S|| = 0.5 -> bound max(1, 0.25)/0.01 = 100 < 101", ([1.0, 101.0], 1, 1.0, 1.0, 0.5, 0.01, 10), 7),
    ("7 takes max(1, .): 50 < 100 (not 0.25/0.01 = 25)", ([1.0, 50.0], 1, 1.0, 1.0, 0.5, 0.01, 10), 0),
    # -- the iteration cap --------------------------------------------------------
    ("8 at k = maxiter = 10",
     ([0.9, 0.8, 0.7, 0.6, 0.5, 0.45, 0.4, 0.35, 0.3, 0.2, 0.1], 10, 1.0, 1.0, 1.0, 0.01, 10), 8),
    ("no 8 at k = 9 < maxiter",
     ([0.9, 0.8, 0.7, 0.6, 0.5, 0.45, 0.4, 0.35, 0.3, 0.2], 9, 1.0, 1.0, 1.0, 0.01, 10), 0),
    # -- condition 5 (maxiter 10: c = 1 + ceil(10/10) = 2; checked at k = 6, 8, 10)
    # A1 = (e2+e3+e4)/2, A2 = (e4+e5+e6)/2 at k = 6
    ("5: A1 = (.22+.29+.21)/2 = .36, A2 = (.21+.24+.21)/2 = .33: .03 >= 1e-4, no stop",
     ([1.0, 0.5, 0.22, 0.29, 0.21, 0.24, 0.21], 6, 1.0, 1.0, 1.0, T4, 10), 0),
    ("5: A1 = (.27+.27+.27)/2 = .405, A2 = (.27+.30+.26)/2 = .415: -.01 < 1e-4",
     ([1.0, 0.5, 0.27, 0.27, 0.27, 0.30, 0.26], 6, 1.0, 1.0, 1.0, T4, 10), 5),
    ("5: A1 = (.30+.26+.30)/2 = .43, A2 = (.30+.28+.29)/2 = .435: -.005 < 1e-4",
     ([1.0, 0.5, 0.30, 0.26, 0.30, 0.28, 0.29], 6, 1.0, 1.0, 1.0, T4, 10), 5),
    ("5 not at k = 2c = 4 (k0 > 2c): A1 = (.27+.27+.27)/2 = .405 < A2 = (.27+.30+.26)/2 = .415 would stop",
     ([0.27, 0.27, 0.27, 0.30, 0.26], 4, 1.0, 1.0, 1.0, T4, 10), 0),
    ("5 not at k = 7 (not a multiple of c = 2)",
     ([1.0, 0.5, 0.4, 0.27, 0.27, 0.27, 0.30, 0.26], 7, 1.0, 1.0, 1.0, T4, 10), 0),
    ("5 at k = 8: A1 = (e4+e5+e6)/2 = .405, A2 = (e6+e7+e8)/2 = .415",
     ([1.0, 0.9, 0.8, 0.7, 0.27, 0.27, 0.27, 0.30, 0.26], 8, 1.0, 1.0, 1.0, T4, 10), 5),
    ("c = 1 + ceil(9/10) = 2: no batch test at k = 3 (c = 1 would stop: (.3+.3)/1 - (.3+.3)/1 = 0)",
     ([0.5, 0.3, 0.3, 0.3002], 3, 1.0, 1.0, 1.0, T4, 9), 0),
    # -- condition 6 at k = 6: I = (|e3-e4| + |e4-e5| + |e5-e6|)/2 < 1e-3 A2 ------
    ("6: I = 3*2e-4/2 = 3e-4 < 1e-3*(.3004+.3002+.3)/2 = 4.503e-4; A1 - A2 = .0502 (no 5)",
     ([1.0, 0.5, 0.4, 0.3006, 0.3004, 0.3002, 0.3], 6, 1.0, 1.0, 1.0, T4, 10), 6),
    ("6: I = 3*1e-3/2 = 1.5e-3 > 1e-3*A2 = 4.515e-4 (1e-2*A2 would stop)",
     ([1.0, 0.5, 0.4, 0.303, 0.302, 0.301, 0.3], 6, 1.0, 1.0, 1.0, T4, 10), 0),
    ("6 window starts at j = k-c: I = (.0096+2e-4+2e-4)/2 = .005 > 4.5e-4",
     ([1.0, 0.5, 0.4, 0.31, 0.3004, 0.3002, 0.3], 6, 1.0, 1.0, 1.0, T4, 10), 0),
    ("6 sums absolute values: I = (.01+.01+2e-4)/2 = .0101 > 1e-3*(.21+.2+.2002)/2",
     ([1.0, 0.5, 0.3, 0.2, 0.21, 0.2, 0.2002], 6, 1.0, 1.0, 1.0, T4, 10), 0),
    ("6 window ends at j = k: I = (3e-4+3e-4+4e-3)/2 = 2.3e-3 > 1e-3*(.3003+.3+.304)/2",
     ([1.0, 0.5, 0.4, 0.3006, 0.3003, 0.3, 0.304], 6, 1.0, 1.0, 1.0, T4, 10), 0),
    ("5 before 6: A1 - A2 = (.3+.3002-.3002-.3)/2 = 0 and I = 2e-4/2 < 4.5e-4",
     ([1.0, 0.5, 0.3, 0.3002, 0.3002, 0.3002, 0.3], 6, 1.0, 1.0, 1.0, T4, 10), 5),
]


@pytest.mark.parametrize("name,args,expected", STOP_CASES, ids=[c[0][:40] for c in STOP_CASES])
def test_stop_reason_hand_built_histories(name, args, expected):
    assert O.stop_reason(*args) == expected, name


def test_window_constant():
    # c = 1 + ceil(maxiter/10) (Sec. 4.1.3, conditions 5 and 6)
    assert O.window_constant(200) == 21
    assert O.window_constant(10) == 2
    assert O.window_constant(9) == 2
    assert O.window_constant(11) == 3
    assert O.window_constant(1) == 2


def test_damping_update_rule():
    # Sec. 4.1.3 "Updates": mu <- 3 mu if g < 0.25, mu <- mu/3 if g > 0.75
    assert O.update_mu(1.0, 0.1) == 3.0
    assert O.update_mu(1.0, -5.0) == 3.0
    assert O.update_mu(1.0, 0.2499) == 3.0
    assert O.update_mu(1.0, 0.25) == 1.0          # not below 0.25
    assert O.update_mu(1.0, 0.5) == 1.0
    assert O.update_mu(1.0, 0.75) == 1.0          # not above 0.75
    assert O.update_mu(0.9, 0.7501) == pytest.approx(0.3, rel=1e-15)
    assert O.update_mu(2.0, 1.7) == pytest.approx(2.0 / 3.0, rel=1e-15)


def test_gain_ratio():
    # actual over predicted decrease (Sec. 3.5.2): (10 - 6) / 8 = 0.5
    assert O.gain_ratio(10.0, 6.0, 8.0) == 0.5
    # an increase of F gives a negative gain: (10 - 12) / 4 = -0.5
    assert O.gain_ratio(10.0, 12.0, 4.0) == -0.5
    # a non-positive predicted decrease is not trusted: gain 0 (then mu x 3)
    assert O.gain_ratio(10.0, 6.0, 0.0) == 0.0
    assert O.gain_ratio(10.0, 6.0, -1.0) == 0.0


def _columns(norms, dims, seed):
    """Factor matrices whose column r has Euclidean norm norms[r]."""
    g = np.random.default_rng(seed)
    out = []
    for I, n in zip(dims, norms):
        W = g.standard_normal((I, len(n)))
        W = W / np.linalg.norm(W, axis=0) * np.asarray(n, dtype=float)
        out.append(W)
    return out


def test_regularizer_and_preconditioner_third_order_formulas():
    # Sec. 4.8, L = 3 with X, Y, Z of column norms
    #   ||X_r|| = (1, 2), ||Y_r|| = (3, 1), ||Z_r|| = (2, 5):
    #   max_r' ||Y_r'|| ||Z_r'|| = max(6, 5) = 6, max ||X|| ||Z|| = max(2, 10) = 10,
    #   max ||X|| ||Y|| = max(3, 2) = 3, overall maximum 10;
    #   gamma_X^(r) = ||Y_r|| ||Z_r|| * 10 = (60, 50)
    #   gamma_Y^(r) = ||X_r|| ||Z_r|| * 10 = (20, 100)
    #   gamma_Z^(r) = ||X_r|| ||Y_r|| * 10 = (30, 20)
    #   D_X entries ||Y_r||^2 ||Z_r||^2 + mu gamma_X^(r), mu = 0.5: (36 + 30, 25 + 25) = (66, 50)
    #   D_Y: ||X_r||^2 ||Z_r||^2 + mu gamma_Y^(r) = (4 + 10, 100 + 50) = (14, 150)
    #   D_Z: ||X_r||^2 ||Y_r||^2 + mu gamma_Z^(r) = (9 + 15, 4 + 10) = (24, 14)
    Ws = _columns([(1, 2), (3, 1), (2, 5)], (4, 3, 5), 0)
    gamma = O.regularizer(Ws)
    np.testing.assert_allclose(gamma[0], [60, 50], rtol=1e-13)
    np.testing.assert_allclose(gamma[1], [20, 100], rtol=1e-13)
    np.testing.assert_allclose(gamma[2], [30, 20], rtol=1e-13)
    M = O.preconditioner(Ws, gamma, 0.5)
    np.testing.assert_allclose(M[0], [66, 50], rtol=1e-13)
    np.testing.assert_allclose(M[1], [14, 150], rtol=1e-13)
    np.testing.assert_allclose(M[2], [24, 14], rtol=1e-13)


def test_regularizer_maximum_over_all_modes():
    # the maximum runs over every mode's products, not only mode l's:
    #   ||X_r|| = (1, 1), ||Y_r|| = (1, 1), ||Z_r|| = (1, 7): products
    #   YZ = (1, 7), XZ = (1, 7), XY = (1, 1); overall maximum 7;
    #   gamma_X = (7, 49), gamma_Y = (7, 49), gamma_Z = (7, 7)
    Ws = _columns([(1, 1), (1, 1), (1, 7)], (3, 3, 3), 1)
    gamma = O.regularizer(Ws)
    np.testing.assert_allclose(gamma[0], [7, 49], rtol=1e-13)
    np.testing.assert_allclose(gamma[1], [7, 49], rtol=1e-13)
    np.testing.assert_allclose(gamma[2], [7, 7], rtol=1e-13)


@pytest.mark.parametrize("dims,R,seed", [((4, 3, 5), 2, 2), ((3, 2, 4, 2), 3, 3)])
def test_preconditioner_is_diag_of_jtj_plus_mu_d(dims, R, seed):
    # M = diag(J^T J) + mu D with diag(J^T J) from the explicit Jacobian
    # (Lemma "partialf"); general L, the reading of Sec. 4.8's closing display
    g = np.random.default_rng(seed)
    Ws = [g.standard_normal((d, R)) for d in dims]
    J = explicit_jacobian(Ws)
    diag = np.diag(J.T @ J)
    gamma = O.regularizer(Ws)
    mu = 0.37
    M = O.preconditioner(Ws, gamma, mu)
    D = np.concatenate([np.repeat(gamma[l], dims[l]) for l in range(len(dims))])
    np.testing.assert_allclose(np.concatenate([np.repeat(M[l], dims[l]) for l in range(len(dims))]),
                               diag + mu * D, rtol=1e-12)


def test_dgn_reports_the_stop_reason_function():
    # the loop stops with the first condition that holds: with tol above the
    # start's error the first iteration stops on condition 1
    T = np.arange(1.0, 25.0).reshape((2, 3, 4), order="F")
    W0 = [np.ones((2, 1)), np.ones((3, 1)), np.ones((4, 1))]
    _, info = O.dgn(T, W0, O.Options(maxiter=3, tol=2.0))
    assert info["stop"] == 1 and info["iters"] == 1
    assert math.isfinite(info["rel_err"])
