"""The block-Jacobi preconditioner on the GPU (cpd_options.precond =
CPD_PRECOND_BLOCK: per mode the exact diagonal block Pi^(l) + mu diag
gamma^(l) of J^T J + mu D, inverted by an FP64 R x R Cholesky factorisation)
against the FP64 oracle run with the same preconditioner: whole solves on the
uncompressed 20^3 workload, a compressed order-3 problem with refinement, and
an order-4 core solved by the cluster solver; fits within 1e-6, factors within
1e-4 after alignment."""
import numpy as np
import pytest

import oracle as O
import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def cpd():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2110_05997_gb300 import build as b
    b.build()
    from paper_2110_05997_gb300 import cpd as m
    m.lib()
    return m


def _check(T, Wg, lg, Wo, lo):
    T64 = T.astype(np.float64)
    fg, fo = O.fit(T64, Wg, lg), O.fit(T64, Wo, lo)
    assert abs(fg - fo) <= 1e-6, (fg, fo)
    c = O.compare_cpd(Wg, lg, Wo, lo)
    assert max(c["mode_err"]) <= 1e-4 and c["lam_err"] <= 1e-4, c


def _np(W, lam):
    return [w.double().cpu().numpy() for w in W], lam.double().cpu().numpy()


def test_block_precond_uncompressed_20cubed(cpd):
    c = synth.c1_plain_dgn()
    T, R, W0 = c["T"], c["R"], c["W0"]
    opts = cpd.cpd_default_options(compress=0, init="given", precond="block")
    W0f = torch.from_numpy(np.concatenate([w.ravel(order="F") for w in W0]).astype(np.float32)).cuda()
    W, lam, info, _ = cpd.cpd_dgn_solve(torch.from_numpy(synth.flat(T)).cuda(), T.shape, R, opts, W0_flat=W0f)
    torch.cuda.synchronize()
    assert info["status"] == 0
    Wo, lo, io = O.cpd(T, R, O.Options(compress=False, init="given", precond="block"), W0=W0)
    _check(T, *_np(W, lam), Wo, lo)


@pytest.mark.parametrize("dims,R,seed,refine", [((50, 45, 40), 5, 142, 10), ((24, 20, 18, 16), 3, 85, 5),
                                                ((30, 28, 26, 24), 12, 7, 3)])
def test_block_precond_compressed_matches_oracle(cpd, dims, R, seed, refine):
    T, _ = synth.planted(seed, dims, R, 0.0, 1e-5, np.float32)
    opts = cpd.cpd_default_options(refine_maxiter=refine, precond="block", init="random", seed=seed)
    W, lam, info, _ = cpd.cpd_dgn_solve(torch.from_numpy(synth.flat(T)).cuda(), T.shape, R, opts)
    torch.cuda.synchronize()
    assert info["status"] == 0
    T64 = T.astype(np.float64)
    Wo, lo, io = O.cpd(T64, R, O.Options(refine_maxiter=refine, precond="block", init="random", seed=seed))
    assert O.fit(T64, Wo, lo) < 1e-4
    _check(T, *_np(W, lam), Wo, lo)
