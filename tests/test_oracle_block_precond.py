"""Pins for the block-Jacobi preconditioner of the oracle (CPU only): its
blocks are the diagonal blocks of J^T J + mu D built from the explicit
Jacobian (the corollary of Sec. 3.5.3: block l is Pi^(l) (x) I); the PCG with
it reaches the dense solution within n steps (App. A); for rank 1 it equals
the diagonal preconditioner, and the whole dGN with it recovers a planted CPD."""
import numpy as np
import pytest

import oracle as O
import synth
from oracle.jacobian import explicit_jacobian, stack


def _problem(dims, R, seed):
    g = np.random.default_rng(seed)
    return g.standard_normal(dims), [g.standard_normal((d, R)) for d in dims]


@pytest.mark.parametrize("dims,R,seed", [((4, 3, 5), 3, 0), ((3, 2, 4, 2), 2, 1)])
def test_blocks_are_the_diagonal_blocks_of_the_regularised_jtj(dims, R, seed):
    _, Ws = _problem(dims, R, seed)
    J = explicit_jacobian(Ws)
    gamma = O.regularizer(Ws)
    mu = 0.41
    A = J.T @ J + mu * np.diag(np.concatenate([np.repeat(gamma[l], dims[l]) for l in range(len(dims))]))
    Pi1, _ = O.pi_matrices(O.grams(Ws))
    Bs, chol = O.block_preconditioner(Pi1, gamma, mu)
    offs = np.cumsum([0] + [d * R for d in dims])
    for l, d in enumerate(dims):
        blk = A[offs[l]:offs[l + 1], offs[l]:offs[l + 1]]
        # vec is column-major (I_l x R): the block is B_l (x) I_{I_l}
        np.testing.assert_allclose(blk, np.kron(Bs[l], np.eye(d)), rtol=1e-12, atol=1e-12)
        np.testing.assert_allclose(chol[l] @ chol[l].T, Bs[l], rtol=1e-12, atol=1e-12)


def test_block_pcg_is_exact_in_n_steps():
    dims, R = (3, 3, 2), 2
    T, Ws = _problem(dims, R, 5)
    J = explicit_jacobian(Ws)
    gamma = O.regularizer(Ws)
    mu = 0.3
    D = np.concatenate([np.repeat(gamma[l], dims[l]) for l in range(3)])
    g = O.neg_gradient(O.residual(T, Ws), Ws)
    x_ref = np.linalg.solve(J.T @ J + mu * np.diag(D), stack(g))
    Pi1, Pi2 = O.pi_matrices(O.grams(Ws))
    _, chol = O.block_preconditioner(Pi1, gamma, mu)
    n = R * sum(dims)
    x, its = O.pcg_block(Ws, Pi1, Pi2, g, gamma, chol, mu, 4 * n, 1e-28)
    np.testing.assert_allclose(stack(x), x_ref, rtol=1e-7, atol=1e-9)
    assert its <= n


def test_rank_one_block_equals_diagonal_preconditioner():
    # R = 1: Pi^(l) is 1 x 1, the block preconditioner is the diagonal one and
    # the two PCG forms give the same iterates
    dims = (4, 5, 3)
    T, Ws = _problem(dims, 1, 7)
    gamma = O.regularizer(Ws)
    mu = 0.2
    g = O.neg_gradient(O.residual(T, Ws), Ws)
    Pi1, Pi2 = O.pi_matrices(O.grams(Ws))
    _, chol = O.block_preconditioner(Pi1, gamma, mu)
    for maxit in (1, 2, 3):
        xb, ib = O.pcg_block(Ws, Pi1, Pi2, g, gamma, chol, mu, maxit, 0.0)
        xd, idg = O.pcg(Ws, Pi1, Pi2, g, gamma, O.preconditioner(Ws, gamma, mu), mu, maxit, 0.0)
        assert ib == idg
        np.testing.assert_allclose(stack(xb), stack(xd), rtol=1e-10, atol=1e-12)


def test_dgn_with_block_preconditioner_recovers_planted_cpd():
    T, Wt = synth.planted(33, (9, 8, 7), 3)
    W, lam, info = O.cpd(T, 3, O.Options(compress=False, init="random", seed=33, tol=1e-16, maxiter=300,
                                         precond="block"))
    assert O.fit(T, W, lam) < 1e-9
    c = O.compare_cpd(W, lam, Wt, None)
    assert max(c["mode_err"]) < 1e-7
