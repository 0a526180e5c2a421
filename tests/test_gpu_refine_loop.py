"""Refinement as a conditional while node of the solve's CUDA graph.

On a non-default stream a solve is captured once and replayed; its
refinement iterations (one pass over T and one step each, Sec. 4.1.3
formulas on the uncompressed tensor) are then the body of a while node
whose condition the step kernel sets, so only the iterations the stop tests
allow are launched.  On the default stream all refine_maxiter + 1 iterations
are launched and the stopped ones exit at once.  Both must give the same
iteration record and the same fit (the passes sum the gradient with
floating-point atomics, so two runs agree to rounding, not bit for bit), and
the graph must launch 3 kernels fewer for every iteration it skips."""
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


def run(cpd, Td, dims, R, opts, stream):
    l0 = cpd.cpd_launch_count()
    if stream is None:
        W, lam, info, _ = cpd.cpd_dgn_solve(Td, dims, R, opts)
    else:
        with torch.cuda.stream(stream):
            W, lam, info, _ = cpd.cpd_dgn_solve(Td, dims, R, opts, stream=stream)
    torch.cuda.synchronize()
    launches = cpd.cpd_launch_count() - l0
    return [w.double().cpu().numpy() for w in W], lam.double().cpu().numpy(), info, launches


KEYS = ("status", "stop", "refine_iters", "refine_stop")


@pytest.mark.parametrize("seed,dims,R,rho,eta,refine,gram,tol", [
    (142, (50, 45, 40), 5, 0.5, 1e-4, 10, "fp32", 1e-6),
    (142, (50, 45, 40), 5, 0.5, 1e-4, 1, "fp32", 1e-6),
    (142, (50, 45, 40), 5, 0.5, 1e-4, 2, "fp32", 1e-6),
    (11, (120, 100, 90), 6, 0.5, 1e-4, 20, "bf16", 1e-6),
    (142, (50, 45, 40), 5, 0.5, 1e-4, 20, "fp32", 1e-1),
    (85, (24, 20, 18, 16), 3, 0.0, 1e-5, 5, "fp32", 1e-6),
])
def test_graph_loop_equals_direct_launches(cpd, seed, dims, R, rho, eta, refine, gram, tol):
    T, _ = synth.planted(seed, dims, R, rho, eta, np.float32)
    Td = torch.from_numpy(synth.flat(T)).cuda()
    opts = cpd.cpd_default_options(refine_maxiter=refine, gram_precision=gram, tol=tol)
    T64 = T.astype(np.float64)
    Wd, ld, infd, nd = run(cpd, Td, dims, R, opts, None)
    assert infd["status"] == 0
    fd = O.fit(T64, Wd, ld)
    st = torch.cuda.Stream()
    for rep in range(2):                     # capture + launch, then replay
        Wg, lg, infg, ng = run(cpd, Td, dims, R, opts, st)
        for k in KEYS:
            assert infd[k] == infg[k], (k, infd[k], infg[k], rep)
        assert abs(O.fit(T64, Wg, lg) - fd) <= 1e-6, rep
        assert abs(infg["refine_rel_err"] - infd["refine_rel_err"]) <= 1e-6, rep
        J = infg["refine_iters"]
        assert 0 <= J <= refine
        assert ng == nd - 3 * (refine - J), (ng, nd, J, refine, rep)
