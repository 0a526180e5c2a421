"""dGN on a large tensor without compression (thesis Sec. 4.9: the uncompressed
CPD of large tensors): every iteration is one pass over T (residual, ||e||^2
and the MTTKRP gradient) plus the on-device step.  The GPU must match the
FP64 oracle's dgn on the same tensor from the same start: the fit within
1e-6 absolute, the factors after permutation/scaling alignment within 1e-4,
and the pass-based route must be the one that ran (no core solve)."""
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


def _solve(cpd, T, R, W0=None, **kw):
    opts = cpd.cpd_default_options(compress=0, **kw)
    Td = torch.from_numpy(synth.flat(T)).cuda()
    W0d = None
    if W0 is not None:
        W0d = torch.from_numpy(np.concatenate([w.astype(np.float32).ravel(order="F") for w in W0])).cuda()
    cpd.cpd_profile_enable(True)
    cpd.cpd_profile_read()                    # clear
    W, lam, info, _ = cpd.cpd_dgn_solve(Td, T.shape, R, opts, W0_flat=W0d)
    torch.cuda.synchronize()
    stages = cpd.cpd_profile_read()
    cpd.cpd_profile_enable(False)
    return [w.double().cpu().numpy() for w in W], lam.double().cpu().numpy(), info, stages


def _unit_aligned_error(Wg, lg, Wo, lo):
    """Largest relative factor difference after matching the rank-one terms
    (lambda sorted both sides) and their signs."""
    R = len(lg)
    err = 0.0
    for l in range(len(Wg)):
        for r in range(R):
            a, b = Wg[l][:, r], Wo[l][:, r]
            s = 1.0 if a @ b >= 0 else -1.0
            err = max(err, float(np.linalg.norm(a - s * b) / np.linalg.norm(b)))
    return err


@pytest.mark.parametrize("dims,R,seed", [((104, 104, 104), 5, 3), ((40, 36, 32, 30), 4, 8)])
def test_full_dgn_random_start_matches_oracle(cpd, dims, R, seed):
    T, _ = synth.planted(seed, dims, R, 0.0, 1e-5, np.float32)
    Wg, lg, info, stages = _solve(cpd, T, R, init="random", seed=seed, maxiter=60, refine_maxiter=0)
    assert "full_start" in stages and "dgn_core" not in stages, stages
    assert info["status"] == 0, info
    T64 = T.astype(np.float64)
    Wo, lo, io = O.cpd(T64, R, O.Options(compress=False, init="random", seed=seed, maxiter=60, refine_maxiter=0))
    fg, fo = O.fit(T64, Wg, lg), O.fit(T64, Wo, lo)
    assert abs(fg - fo) <= 1e-6, (fg, fo, info)
    assert _unit_aligned_error(Wg, lg, Wo, lo) <= 1e-4


def test_full_dgn_given_start_then_refinement(cpd):
    dims, R = (110, 100, 96), 6
    T, Wt = synth.planted(21, dims, R, 0.3, 1e-6, np.float32)
    g = np.random.default_rng(5)
    W0 = [w + 0.05 * g.standard_normal(w.shape) for w in Wt]
    Wg, lg, info, stages = _solve(cpd, T, R, W0=W0, init="given", maxiter=8, refine_maxiter=4)
    assert "full_start" in stages
    assert info["status"] == 0 and info["iters"] >= 1, info
    T64 = T.astype(np.float64)
    W0_32 = [w.astype(np.float32).astype(np.float64) for w in W0]
    Wo, lo, io = O.cpd(T64, R, O.Options(compress=False, init="given", maxiter=8, refine_maxiter=4), W0=W0_32)
    fg, fo = O.fit(T64, Wg, lg), O.fit(T64, Wo, lo)
    assert abs(fg - fo) <= 1e-6, (fg, fo, info)
