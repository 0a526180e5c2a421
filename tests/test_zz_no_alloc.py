"""cpd_dgn_solve_noalloc: the workspace-free variant of the uncompressed dGN
solve, for callers that may not allocate device memory when they need a CPD.
Its scratch is a fixed device array inside the library; this test calls it
twice in a row through the C ABI and checks both results against the regular
cpd_dgn_solve on the same input, with the tolerances of the other parity
tests (fit within 1e-6 absolute, factors within 1e-4 after alignment).  The
file name makes pytest collect it last; it also passes on its own in a fresh
process."""
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


def _np(W, lam):
    return [w.double().cpu().numpy() for w in W], lam.double().cpu().numpy()


def test_noalloc_matches_workspace_solve_twice(cpd):
    c = synth.c1_plain_dgn()
    T, R, W0 = c["T"], c["R"], c["W0"]
    Tf = torch.from_numpy(synth.flat(T)).cuda()
    W0f = torch.from_numpy(np.concatenate([w.ravel(order="F") for w in W0]).astype(np.float32)).cuda()
    opts = cpd.cpd_default_options(compress=0, init="given")
    Wr, lr, ir, _ = cpd.cpd_dgn_solve(Tf, T.shape, R, opts, W0_flat=W0f)
    torch.cuda.synchronize()
    Wr, lr = _np(Wr, lr)
    fr = O.fit(T, Wr, lr)
    for call in range(2):
        W, lam, info = cpd.cpd_dgn_solve_noalloc(Tf, T.shape, R, opts, W0_flat=W0f)
        torch.cuda.synchronize()
        Wn, ln = _np(W, lam)
        assert info["status"] == 0 and info["iters"] == ir["iters"], (call, info, ir)
        assert abs(O.fit(T, Wn, ln) - fr) <= 1e-6, call
        cmp_ = O.compare_cpd(Wn, ln, Wr, lr)
        assert max(cmp_["mode_err"]) <= 1e-4 and cmp_["lam_err"] <= 1e-4, (call, cmp_)


def test_noalloc_refuses_problems_beyond_its_capacity(cpd):
    T, _ = synth.planted(4, (10, 10, 10), 2)
    Tf = torch.from_numpy(synth.flat(T)).cuda()
    with pytest.raises(cpd.CpdError) as e:
        cpd.cpd_dgn_solve_noalloc(Tf, T.shape, 2, cpd.cpd_default_options(compress=0, init="random",
                                                                          maxiter=5000))
    assert e.value.status == -3
    with pytest.raises(cpd.CpdError) as e:
        cpd.cpd_dgn_solve_noalloc(Tf, T.shape, 2, cpd.cpd_default_options(init="random"))   # compress = 1
    assert e.value.status == -6
