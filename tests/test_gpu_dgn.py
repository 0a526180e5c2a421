"""GPU parity of the on-core damped Gauss-Newton (C ABI) against the FP64 oracle.

Tolerances: the CUDA path computes in FP32 with FP64 scalar recurrences; a
single FP32 pass (residual, MTTKRP, J^T J v) is compared entry by entry with
relative error 2e-5 of the vector norm (FP32 unit roundoff 6e-8 times the
summation lengths here, with margin).  Whole solves are compared on what is
unique: the fit scored by the oracle's FP64 evaluator (within 1e-6 absolute)
and the factors after permutation/scaling alignment (within 1e-4 relative).
"""
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


def dev(x, dtype=np.float32):
    return torch.from_numpy(np.ascontiguousarray(x, dtype=dtype)).cuda()


def stacked(Ws):
    return np.concatenate([np.asarray(W).ravel(order="F") for W in Ws])


def unstack(w, dims, R):
    out, o = [], 0
    for d in dims:
        out.append(np.asarray(w[o:o + d * R]).reshape((d, R), order="F"))
        o += d * R
    return out


SHAPES = [((5, 4, 3), 2), ((20, 20, 20), 5), ((3, 17, 5), 4), ((33, 2, 7), 3), ((2, 2, 2), 1),
          ((7, 9, 5, 6), 3), ((4, 3, 5, 2), 2), ((10, 10, 10), 10)]


@pytest.mark.parametrize("dims,R", SHAPES)
def test_core_eval_matches_oracle(cpd, dims, R):
    g = np.random.default_rng(sum(dims) * 31 + R)
    S = g.standard_normal(dims).astype(np.float32).astype(np.float64)
    Ws = [g.standard_normal((d, R)).astype(np.float32).astype(np.float64) for d in dims]
    f, gr, fsq = cpd.cpd_core_eval(dev(synth.flat(S)), dims, R, dev(stacked(Ws)))
    torch.cuda.synchronize()
    f_or = O.residual(S, Ws)
    g_or = stacked(O.neg_gradient(f_or, Ws))
    np.testing.assert_allclose(f.cpu().numpy(), synth.flat(f_or), rtol=0,
                               atol=2e-5 * max(1.0, np.abs(f_or).max()))
    assert abs(fsq.item() - np.sum(f_or ** 2)) <= 2e-5 * np.sum(f_or ** 2)
    assert np.linalg.norm(gr.cpu().numpy() - g_or) <= 2e-5 * np.linalg.norm(g_or) + 1e-6


@pytest.mark.parametrize("dims,R", SHAPES)
def test_jtj_apply_matches_oracle(cpd, dims, R):
    g = np.random.default_rng(sum(dims) * 17 + R)
    Ws = [g.standard_normal((d, R)).astype(np.float32).astype(np.float64) for d in dims]
    Vs = [g.standard_normal((d, R)).astype(np.float32).astype(np.float64) for d in dims]
    out = cpd.cpd_jtj_apply(dims, R, dev(stacked(Ws)), dev(stacked(Vs)))
    torch.cuda.synchronize()
    Pi1, Pi2 = O.pi_matrices(O.grams(Ws))
    ref = stacked(O.jtj_apply(Ws, Pi1, Pi2, Vs))
    assert np.linalg.norm(out.cpu().numpy() - ref) <= 2e-5 * np.linalg.norm(ref)


def _solve_uncompressed(cpd, T, R, W0, maxiter=200, trace=False, tol=1e-6, threads=0):
    opts = cpd.cpd_default_options(compress=0, init="given", maxiter=maxiter, tol=tol,
                                   block_threads=threads)
    Tf = dev(synth.flat(T), np.float64 if T.dtype == np.float64 else np.float32)
    W, lam, info, tr = cpd.cpd_dgn_solve(Tf, T.shape, R, opts, W0_flat=dev(stacked(W0)), trace=trace)
    torch.cuda.synchronize()
    return ([w.double().cpu().numpy() for w in W], lam.double().cpu().numpy(), info,
            None if tr is None else tr.cpu().numpy())


def test_dgn_plain_20cubed_rank5_fp64(cpd):
    """The plain-dGN workload (20x20x20 FP64, rank 5, noise 1e-6, N(0,1) start)."""
    c = synth.c1_plain_dgn()
    T, R, W0 = c["T"], c["R"], c["W0"]
    Wg, lg, info, _ = _solve_uncompressed(cpd, T, R, W0)
    assert info["status"] == 0 and 1 <= info["stop"] <= 8
    Wo, lo, io = O.cpd(T, R, O.Options(compress=False, init="given"), W0=W0)
    fg, fo = O.fit(T, Wg, lg), O.fit(T, Wo, lo)
    assert abs(fg - fo) <= 1e-6, (fg, fo, info, io)
    cmp_ = O.compare_cpd(Wg, lg, Wo, lo)
    assert max(cmp_["mode_err"]) <= 1e-4 and cmp_["lam_err"] <= 1e-4, cmp_
    # and both found the planted CPD
    cmp_t = O.compare_cpd(Wg, lg, c["W_true"], None)
    assert max(cmp_t["mode_err"]) <= 1e-4


def test_dgn_first_iterations_track_oracle(cpd):
    c = synth.c1_plain_dgn()
    T, R, W0 = c["T"], c["R"], c["W0"]
    _, _, info, tr = _solve_uncompressed(cpd, T, R, W0, maxiter=4, trace=True, tol=0.0)
    otr = []
    O.dgn(T, W0, O.Options(compress=False, maxiter=4, tol=0.0), trace=otr)
    for k in range(3):
        g, o = tr[k], otr[k]
        assert int(g[0]) == o["k"]
        assert int(g[4]) == o["cg"]                      # same cg_maxiter draw, no early exit
        assert abs(g[1] - o["rel_err"]) <= 1e-3 * o["rel_err"]
        assert abs(g[2] - o["mu"]) <= 1e-6 * o["mu"]     # mu moves by exact factors of 3
        assert abs(g[5] - o["step"]) <= 1e-3 * o["step"]


@pytest.mark.parametrize("dims,R,seed", [((6, 5, 4), 1, 1), ((3, 17, 5), 2, 2), ((9, 8, 7, 6), 3, 3),
                                         ((2, 2, 2), 1, 4), ((40, 6, 3), 3, 5)])
def test_dgn_edge_shapes_recover_planted(cpd, dims, R, seed):
    T, Wt = synth.planted(seed + 100, dims, R, 0.0, 1e-7)
    W0 = synth.initial_factors(seed, dims, R)
    Wg, lg, info, _ = _solve_uncompressed(cpd, T, R, W0, maxiter=300)
    Wo, lo, io = O.cpd(T, R, O.Options(compress=False, init="given", maxiter=300), W0=W0)
    fg, fo = O.fit(T, Wg, lg), O.fit(T, Wo, lo)
    assert abs(fg - fo) <= 1e-6, (fg, fo, info, io)


@pytest.mark.parametrize("threads", [64, 128, 512, 1024])
def test_dgn_block_size_does_not_change_the_answer(cpd, threads):
    c = synth.c1_plain_dgn()
    Wg, lg, info, _ = _solve_uncompressed(cpd, c["T"], c["R"], c["W0"], threads=threads)
    Wo, lo, io = O.cpd(c["T"], c["R"], O.Options(compress=False, init="given"), W0=c["W0"])
    assert abs(O.fit(c["T"], Wg, lg) - O.fit(c["T"], Wo, lo)) <= 1e-6


def test_dgn_random_init_matches_oracle_draws(cpd):
    # INIT_RANDOM draws the same N(0,1) numbers on both sides (SplitMix64 + Box-Muller)
    T, Wt = synth.planted(77, (8, 7, 6), 2, 0.0, 1e-7)
    opts = cpd.cpd_default_options(compress=0, init="random", seed=5, maxiter=1, tol=0.0)
    W, lam, info, tr = cpd.cpd_dgn_solve(dev(synth.flat(T)), T.shape, 2, opts, trace=True)
    otr = []
    O.dgn(T, O.init_random(5, T.shape, 2), O.Options(maxiter=1, tol=0.0, seed=5), trace=otr)
    torch.cuda.synchronize()
    g = tr.cpu().numpy()[0]
    assert abs(g[1] - otr[0]["rel_err"]) <= 1e-4 * otr[0]["rel_err"]


def test_nan_input_reports_numeric_status(cpd):
    T, _ = synth.planted(3, (5, 5, 5), 2)
    T[1, 2, 3] = np.nan
    W0 = synth.initial_factors(3, T.shape, 2)
    Wg, lg, info, _ = _solve_uncompressed(cpd, T, 2, W0, maxiter=10)
    assert info["status"] == -4
