"""Pins for the oracle's damped Gauss-Newton (CPU only): gradient against
brute-force sums and finite differences, J^T J·v against an explicit
Jacobian, PCG against a dense solve, the regulariser's stated purpose,
SplitMix64 reference outputs, and end-to-end recovery."""
import itertools
import math

import numpy as np
import pytest

import oracle as O
import synth
from oracle.jacobian import explicit_jacobian, stack, unstack


def _rand_problem(dims, R, seed=0):
    g = np.random.default_rng(seed)
    T = g.standard_normal(dims)
    Ws = [g.standard_normal((d, R)) for d in dims]
    return T, Ws


def _F(T, Ws):
    f = O.residual(T, Ws)
    return 0.5 * float(np.sum(f * f))


@pytest.mark.parametrize("dims,R", [((4, 3, 2), 2), ((3, 2, 3, 2), 2)])
def test_gradient_brute_force_and_finite_differences(dims, R):
    T, Ws = _rand_problem(dims, R, 1)
    f = O.residual(T, Ws)
    g = O.neg_gradient(f, Ws)
    L = len(dims)
    # Theorem "partialF" written as the brute-force sum of Sec. 3.4 (after Lemma partialf)
    for lp in range(L):
        for ip in range(dims[lp]):
            for rp in range(R):
                s = 0.0
                for idx in itertools.product(*[range(d) for d in dims]):
                    if idx[lp] != ip:
                        continue
                    resid = T[idx] - sum(np.prod([Ws[l][idx[l], r] for l in range(L)]) for r in range(R))
                    s += resid * np.prod([Ws[l][idx[l], rp] for l in range(L) if l != lp])
                assert abs(g[lp][ip, rp] - s) < 1e-10
    # central finite differences of F: dF/dw = -g
    h = 1e-6
    for lp in range(L):
        for ip, rp in [(0, 0), (dims[lp] - 1, R - 1)]:
            Wp = [W.copy() for W in Ws]
            Wm = [W.copy() for W in Ws]
            Wp[lp][ip, rp] += h
            Wm[lp][ip, rp] -= h
            fd = (_F(T, Wp) - _F(T, Wm)) / (2 * h)
            assert abs(fd + g[lp][ip, rp]) < 1e-6 * max(1.0, abs(fd))


def test_gradient_kolda_form():
    # dF/dW^(l) = W^(l)Pi^(l) - T_(l)·KR (Sec. 4.1.3): same as -f_(l)·KR
    T, Ws = _rand_problem((5, 4, 3), 3, 2)
    g = O.neg_gradient(O.residual(T, Ws), Ws)
    Pi1, _ = O.pi_matrices(O.grams(Ws))
    from oracle.tensor import kr_others
    for l in range(3):
        dF = Ws[l] @ Pi1[l] - O.unfold(T, l) @ kr_others(Ws, l)
        np.testing.assert_allclose(-g[l], dF, atol=1e-10)


@pytest.mark.parametrize("dims,R,seed", [((4, 3, 2), 2, 0), ((3, 4, 2, 3), 3, 1), ((5, 2, 3), 4, 2)])
def test_jtj_apply_against_explicit_jacobian(dims, R, seed):
    # Theorem "Hv" vs J^T J built from Lemma "partialf"; (4,3,2), R=2 is the
    # thesis's own illustration of J's structure (Fig. structure-concrete)
    _, Ws = _rand_problem(dims, R, seed)
    J = explicit_jacobian(Ws)
    JtJ = J.T @ J
    g = np.random.default_rng(seed + 10)
    Vs = [g.standard_normal((d, R)) for d in dims]
    Pi1, Pi2 = O.pi_matrices(O.grams(Ws))
    hv = stack(O.jtj_apply(Ws, Pi1, Pi2, Vs))
    np.testing.assert_allclose(hv, JtJ @ stack(Vs), rtol=1e-11, atol=1e-11)
    # Theorem "JfT_Jf": diagonal blocks are Pi^(l') ⊗ I
    offs = np.cumsum([0] + [d * R for d in dims])
    for l in range(len(dims)):
        blk = JtJ[offs[l]:offs[l + 1], offs[l]:offs[l + 1]]
        np.testing.assert_allclose(blk, np.kron(Pi1[l], np.eye(dims[l])), atol=1e-11)
    # J^T f = grad F = -(A^T b)
    T = np.random.default_rng(seed + 20).standard_normal(dims)
    f = O.residual(T, Ws)
    np.testing.assert_allclose(J.T @ f.ravel(order="F"), -stack(O.neg_gradient(f, Ws)), atol=1e-10)


def test_jtj_scaling_null_vectors():
    # Theorem "J^T J is singular": scaling term r by (1+t) in mode 1 and by
    # 1/(1+t) in mode 2 leaves the tensor fixed, so v = (w_r^(1), -w_r^(2), 0) ∈ ker J
    dims, R = (4, 3, 5), 2
    _, Ws = _rand_problem(dims, R, 3)
    Pi1, Pi2 = O.pi_matrices(O.grams(Ws))
    for r in range(R):
        Vs = [np.zeros((d, R)) for d in dims]
        Vs[0][:, r] = Ws[0][:, r]
        Vs[1][:, r] = -Ws[1][:, r]
        hv = stack(O.jtj_apply(Ws, Pi1, Pi2, Vs))
        assert np.linalg.norm(hv) < 1e-10 * np.linalg.norm(stack(Ws)) ** 3


def test_regularizer_makes_system_diagonally_dominant():
    # Sec. 4.8: J^T J + D is diagonally dominant; the a_ii part of M is diag(J^T J)
    dims, R = (4, 3, 3), 3
    _, Ws = _rand_problem(dims, R, 4)
    J = explicit_jacobian(Ws)
    JtJ = J.T @ J
    gamma = O.regularizer(Ws)
    D = np.concatenate([np.repeat(gamma[l], dims[l]) for l in range(3)])
    A = JtJ + np.diag(D)
    off = np.sum(np.abs(A), axis=1) - np.abs(np.diag(A))
    assert np.all(np.diag(A) >= np.max(np.abs(A - np.diag(np.diag(A))), axis=1) - 1e-12)
    M0 = O.preconditioner(Ws, gamma, 0.0)
    np.testing.assert_allclose(np.concatenate([np.repeat(M0[l], dims[l]) for l in range(3)]),
                               np.diag(JtJ), rtol=1e-12)
    mu = 0.7
    M = O.preconditioner(Ws, gamma, mu)
    np.testing.assert_allclose(np.concatenate([np.repeat(M[l], dims[l]) for l in range(3)]),
                               np.diag(JtJ) + mu * D, rtol=1e-12)
    assert off.shape == D.shape


def test_pcg_is_exact_in_n_steps():
    # App. A: CG reaches the exact solution in at most n steps
    dims, R = (3, 3, 2), 2
    T, Ws = _rand_problem(dims, R, 5)
    J = explicit_jacobian(Ws)
    gamma = O.regularizer(Ws)
    mu = 0.3
    D = np.concatenate([np.repeat(gamma[l], dims[l]) for l in range(3)])
    g = O.neg_gradient(O.residual(T, Ws), Ws)
    x_ref = np.linalg.solve(J.T @ J + mu * np.diag(D), stack(g))
    Pi1, Pi2 = O.pi_matrices(O.grams(Ws))
    n = R * sum(dims)
    x, its = O.pcg(Ws, Pi1, Pi2, g, gamma, O.preconditioner(Ws, gamma, mu), mu, 4 * n, 1e-28)
    np.testing.assert_allclose(stack(x), x_ref, rtol=1e-7, atol=1e-9)


def test_splitmix64_reference_outputs():
    # published SplitMix64 outputs (state 0 and state 1234567)
    assert O.splitmix64(0, 0, 1) == 0xE220A8397B1DCDAF
    expect = [6457827717110365317, 3203168211198807973, 9817491932198370423,
              4593380528125082431, 16408922859458223821]
    assert [O.splitmix64(1234567, 0, c) for c in range(1, 6)] == expect


def test_cg_maxiter_interval_and_spread():
    for k in list(range(1, 300)) + [1000, 5000]:
        lo = 1 + math.ceil(k ** 0.4 - 1e-9)
        hi = 2 + math.ceil(k ** 0.9 - 1e-9)
        v = O.cg_maxiter(k, 42)
        assert lo <= v <= hi
    # k = 32: 32^0.4 = 4 exactly, so the interval starts at 5, not 6
    vals = {O.cg_maxiter(32, s) for s in range(400)}
    assert min(vals) == 5 and max(vals) == 2 + math.ceil(32 ** 0.9 - 1e-9)
    # roughly uniform over a wide interval
    k = 200
    lo, hi = 1 + math.ceil(k ** 0.4), 2 + math.ceil(k ** 0.9)
    draws = np.array([O.cg_maxiter(k, s) for s in range(20000)])
    counts = np.bincount(draws - lo, minlength=hi - lo + 1)
    exp = len(draws) / (hi - lo + 1)
    chi2 = float(np.sum((counts - exp) ** 2 / exp))
    assert chi2 < 2 * (hi - lo + 1)


def test_init_random_is_standard_normal():
    Ws = O.init_random(9, (60, 50), 20)
    x = np.concatenate([W.ravel() for W in Ws])
    assert abs(x.mean()) < 0.05 and abs(x.std() - 1) < 0.05
    assert abs(np.mean(x ** 4) - 3) < 0.3


def test_balance_keeps_tensor_and_equalises_norms():
    _, Ws = _rand_problem((4, 5, 6), 3, 6)
    B = O.balance(Ws)
    np.testing.assert_allclose(O.cpd_tensor(B), O.cpd_tensor(Ws), atol=1e-12)
    nr = np.array([np.linalg.norm(W, axis=0) for W in B])
    np.testing.assert_allclose(nr, nr[0:1].repeat(3, 0), rtol=1e-12)
    for W0, W1 in zip(Ws, B):
        assert np.all(np.sign(W0) == np.sign(W1))


def test_dgn_descent_and_gain_denominator():
    # Theorem (dGN) item 2 and the gain-ratio denominator > 0 (Sec. 3.5.2): along a
    # run, <grad F, x> < 0 and F - ½||f + Jx||^2 = ||Jx||^2 + ... > 0
    T, _ = synth.planted(21, (6, 5, 4), 3, 0.0, 0.01)
    Ws = O.balance(O.init_random(3, T.shape, 3))
    mu = float(np.mean(np.abs(T)))
    for k in range(1, 8):
        f = O.residual(T, Ws)
        g = O.neg_gradient(f, Ws)
        gr = O.grams(Ws)
        Pi1, Pi2 = O.pi_matrices(gr)
        gamma = O.regularizer(Ws)
        x, _ = O.pcg(Ws, Pi1, Pi2, g, gamma, O.preconditioner(Ws, gamma, mu), mu,
                     O.cg_maxiter(k, 0), 1e-6)
        J = explicit_jacobian(Ws)
        xs = stack(x)
        assert float(stack(g) @ xs) > 0          # <grad F, x> < 0
        pred = 0.5 * np.sum((f.ravel(order="F") + J @ xs) ** 2)
        F = 0.5 * np.sum(f * f)
        assert F - pred > 0
        Hx = O.jtj_apply(Ws, Pi1, Pi2, x)
        assert abs((F - pred) - (float(stack(g) @ xs) - 0.5 * float(stack(Hx) @ xs))) < 1e-9 * F
        Ws = O.balance([W + X for W, X in zip(Ws, x)])


@pytest.mark.parametrize("dims,R,seed", [((9, 8, 7), 3, 31), ((6, 5, 4, 5), 2, 32)])
def test_dgn_recovers_planted_noiseless(dims, R, seed):
    T, Wt = synth.planted(seed, dims, R)
    W, lam, info = O.cpd(T, R, O.Options(compress=False, init="random", seed=seed,
                                          tol=1e-16, maxiter=300))
    assert O.fit(T, W, lam) < 1e-9
    cmp_ = O.compare_cpd(W, lam, Wt, None)
    assert max(cmp_["mode_err"]) < 1e-7 and cmp_["lam_err"] < 1e-7


def test_warming_up_exact_recovery():
    # Sec. 4.2: the columns of the computed factors are multiples of the
    # separable functions cos(1-x), -sin(1+x^2)e^{x^2}, -cos(x), ...
    T = synth.warming_up_tensor()
    W, lam, info = O.cpd(T, 3, O.Options(tol=1e-14))
    assert O.fit(T, W, lam) < 1e-6
    cmp_ = O.compare_cpd(W, lam, synth.warming_up_separable(), None)
    assert max(cmp_["mode_err"]) < 2e-4


def test_compressed_path_matches_uncompressed_optimum():
    # compression is exact for a noiseless rank-R tensor (Remark "mlsvd-cpd")
    T, Wt = synth.planted(41, (12, 11, 10), 3)
    W, lam, info = O.cpd(T, 3, O.Options(tol=1e-16, maxiter=300, init="mlsvd"))
    assert info["core_dims"] == [3, 3, 3]
    assert O.fit(T, W, lam) < 1e-9


def test_normalize_reconstructs_and_sorts():
    _, Ws = _rand_problem((4, 5, 6), 4, 7)
    Wn, lam = O.normalize(Ws)
    np.testing.assert_allclose(O.cpd_tensor(Wn, lam), O.cpd_tensor(Ws), atol=1e-10)
    assert np.all(np.diff(lam) <= 0)
    for W in Wn:
        np.testing.assert_allclose(np.linalg.norm(W, axis=0), 1.0, rtol=1e-12)


def test_align_recovers_permutation_and_scaling():
    _, Ws = _rand_problem((5, 4, 6), 4, 8)
    perm = np.array([2, 0, 3, 1])
    sc = [np.array([2.0, -1.0, 0.5, 3.0]), np.array([1.0, 4.0, -2.0, 1.0])]
    Wb = [Ws[0][:, perm] * sc[0], Ws[1][:, perm] * sc[1], Ws[2][:, perm] / (sc[0] * sc[1])]
    c = O.compare_cpd(Ws, None, Wb, None)
    assert max(c["mode_err"]) < 1e-12 and c["lam_err"] < 1e-12


def test_stop_conditions_order_and_windows():
    # maxiter cap and the window constant c = 1 + ceil(maxiter/10)
    T, _ = synth.planted(51, (7, 6, 5), 2, 0.0, 0.05)
    W, info = O.dgn(T, O.init_random(5, T.shape, 2), O.Options(maxiter=5, tol=0.0))
    assert info["iters"] == 5 and info["stop"] == 8
    # a tolerance above the initial error stops at iteration 1 on test 1
    W, info = O.dgn(T, O.init_random(5, T.shape, 2), O.Options(maxiter=50, tol=10.0))
    assert info["iters"] == 1 and info["stop"] == 1
