"""cpd_dgn_solve_noalloc: the workspace-free variant of the uncompressed dGN
solve, for callers that may not allocate device memory when they need a CPD.
Its scratch is a fixed device array inside the library; this test calls it
twice in a row through the C ABI and checks both results against the regular
cpd_dgn_solve on the same input and against the FP64 oracle, with the
tolerances of the other parity tests (fit within 1e-6 absolute, factors within
1e-4 after alignment), on a problem whose CTA keeps one unknown per thread
and on one with more unknowns (1056) than threads.  The file name makes
pytest collect it last; it also passes on its own in a fresh process."""
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


def _problem(which):
    if which == "20x20x20_r5":
        c = synth.c1_plain_dgn()
        return c["T"], c["R"], c["W0"], 1e-6
    # 16 * (30 + 24 + 12) = 1056 unknowns: more than one CTA's 1024 threads;
    # the start is the planted factors plus 10 % Gaussian perturbation
    T, Wt = synth.planted(77, (30, 24, 12), 16, 0.0, 1e-6)
    g = np.random.default_rng(78)
    W0 = [w + 0.1 * g.standard_normal(w.shape) * np.linalg.norm(w, axis=0) / np.sqrt(w.shape[0]) for w in Wt]
    return T, 16, W0, 1e-8     # tol below the noise: both sides run to the noise floor


@pytest.mark.parametrize("which", ["20x20x20_r5", "30x24x12_r16"])
def test_noalloc_matches_workspace_solve_and_oracle_twice(cpd, which):
    T, R, W0, tol = _problem(which)
    Tf = torch.from_numpy(synth.flat(T)).cuda()
    W0f = torch.from_numpy(np.concatenate([w.ravel(order="F") for w in W0]).astype(np.float32)).cuda()
    opts = cpd.cpd_default_options(compress=0, init="given", tol=tol)
    Wr, lr, ir, _ = cpd.cpd_dgn_solve(Tf, T.shape, R, opts, W0_flat=W0f)
    torch.cuda.synchronize()
    Wr, lr = _np(Wr, lr)
    fr = O.fit(T, Wr, lr)
    Wo, lo, io = O.cpd(T, R, O.Options(compress=False, init="given", tol=tol), W0=W0)
    fo = O.fit(T, Wo, lo)
    assert fo < 1e-5
    for call in range(2):
        W, lam, info = cpd.cpd_dgn_solve_noalloc(Tf, T.shape, R, opts, W0_flat=W0f)
        torch.cuda.synchronize()
        Wn, ln = _np(W, lam)
        assert info["status"] == 0 and info["iters"] == ir["iters"], (call, info, ir)
        fn = O.fit(T, Wn, ln)
        assert abs(fn - fr) <= 1e-6, call
        assert abs(fn - fo) <= 1e-6, (call, fn, fo)
        for ref in ((Wr, lr), (Wo, lo)):
            cmp_ = O.compare_cpd(Wn, ln, *ref)
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
