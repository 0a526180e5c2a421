"""GPU parity of the batched solver (one persistent launch, one CTA per CPD)
against the FP64 oracle run item by item with the same options and seeds.

The bar, per item, with "solved" meaning a fit below 10x the noise level:
  * an item both sides solve has |fit_GPU - fit_oracle| <= 1e-6 (both scored by
    the oracle's FP64 evaluator) and factors within 1e-4 after alignment;
  * dGN converges to a local minimum (Sec. 3.5) and some starts lead into one
    (Sec. 4.1.2); starts that agree to FP32 rounding can end at different
    stationary points, so an item can stall on one side only.  Items that stall
    on the GPU only must be no more frequent than items that stall in the
    oracle only (on the 1024-item sample; small cases allow one item of
    sampling slack), and every item ends with a normal stop.
These workloads have noise eta = 1e-6.  With the stop tolerance at the noise
level (tol = 1e-6) the improvement test |e_{k-1} - e_k| < tol fires at an
iteration that depends on rounding, above the noise floor, and 1 % of the
items then differ from the oracle by up to 2e-6; the batched workload is
therefore run with tol = 1e-7, one decade below the noise, on both sides."""
import os

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


def pack(items):
    offs, o = [], 0
    for it in items:
        offs.append(o)
        o += it["T"].size
    flat = np.concatenate([synth.flat(it["T"]).astype(np.float32) for it in items])
    return torch.from_numpy(flat).cuda(), offs


def unpack(W, lam, w_off, l_off, dims, R):
    Ws, o = [], w_off
    w = W[o:o + R * sum(dims)].double().cpu().numpy()
    k = 0
    for d in dims:
        Ws.append(w[k:k + d * R].reshape((d, R), order="F"))
        k += d * R
    return Ws, lam[l_off:l_off + R].double().cpu().numpy()


def run_batch(cpd, items, **kw):
    Tp, offs = pack(items)
    dims = [list(it["T"].shape) for it in items]
    ranks = [it["R"] for it in items]
    opts = cpd.cpd_default_options(**kw)
    W, lam, w_off, l_off, infos = cpd.cpd_batch_solve(Tp, offs, dims, ranks, opts)
    torch.cuda.synchronize()
    return [unpack(W, lam, w_off[b], l_off[b], dims[b], ranks[b]) for b in range(len(items))], infos


TOL = 1e-7


def check_item(it, Wg, lg, seed, rel_eta, tol=TOL):
    """"both" (after asserting the fit and factor bar) when both sides solve
    the item, "oracle_only" / "gpu_only" when only that side stalls, None when
    both stall."""
    T = it["T"].astype(np.float64)
    Wo, lo, io = O.cpd(T, it["R"], O.Options(seed=int(seed), tol=tol))
    return judge(T, it["R"], Wg, lg, Wo, lo, rel_eta)


def judge(T, R, Wg, lg, Wo, lo, rel_eta):
    fo, fg = O.fit(T, Wo, lo), O.fit(T, Wg, lg)
    so, sg = fo >= 10 * rel_eta, fg >= 10 * rel_eta
    if so and sg:
        return None
    if so:
        return "oracle_only"
    if sg:
        return "gpu_only"
    assert abs(fg - fo) <= 1e-6, (fg, fo, T.shape, R)
    c = O.compare_cpd(Wg, lg, Wo, lo)
    assert max(c["mode_err"]) <= 1e-4 and c["lam_err"] <= 1e-4, c
    return "both"


def summarize(results, min_solved, slack=1):
    n = len(results)
    both = results.count("both")
    go, oo = results.count("gpu_only"), results.count("oracle_only")
    assert both >= min_solved * n, (both, n)
    assert go <= oo + slack, (go, oo)


def test_batch_small_uneven_matches_oracle(cpd):
    items = synth.c4_batch(seed=7, B=48, lo=6, hi=20, rlo=1, rhi=6, eta=1e-6)
    res, infos = run_batch(cpd, items, seed=11, tol=TOL)
    out = []
    for b, (it, (Wg, lg)) in enumerate(zip(items, res)):
        assert infos[b]["status"] == 0
        out.append(check_item(it, Wg, lg, 11 + b, 1e-6))
    summarize(out, 0.75)


def test_batch_equals_single_solves(cpd):
    items = synth.c4_batch(seed=8, B=6, lo=8, hi=30, rlo=2, rhi=8, eta=1e-6)
    res, infos = run_batch(cpd, items, seed=3)
    for b, it in enumerate(items):
        T = it["T"]
        opts = cpd.cpd_default_options(seed=3 + b)
        W, lam, info, _ = cpd.cpd_dgn_solve(torch.from_numpy(synth.flat(T)).cuda(), T.shape, it["R"], opts)
        torch.cuda.synchronize()
        Ws = [w.double().cpu().numpy() for w in W]
        ls = lam.double().cpu().numpy()
        T64 = T.astype(np.float64)
        assert abs(O.fit(T64, Ws, ls) - O.fit(T64, *res[b])) <= 1e-6
        assert infos[b]["core_dims"][:3] == info["core_dims"][:3]


def test_batch_edge_shapes(cpd):
    rng = np.random.default_rng(0)
    shapes = [((2, 2, 2), 1), ((2, 9, 3), 2), ((64, 3, 5), 3), ((5, 64, 64), 4), ((7, 7, 7), 7)]
    items = []
    for i, (dims, R) in enumerate(shapes):
        T, Wt = synth.planted(500 + i, dims, R, 0.0, 1e-6, np.float32)
        items.append(dict(T=T, R=R, W_true=Wt))
    res, infos = run_batch(cpd, items, seed=1, tol=TOL)
    out = []
    for b, it in enumerate(items):
        assert infos[b]["status"] == 0
        out.append(check_item(it, *res[b], 1 + b, 1e-6))
    summarize(out, 0.6)


def test_batch_uncompressed(cpd):
    items = synth.c4_batch(seed=9, B=8, lo=4, hi=9, rlo=1, rhi=3, eta=1e-6)
    res, infos = run_batch(cpd, items, seed=2, compress=0, tol=TOL)
    out = []
    for b, it in enumerate(items):
        assert infos[b]["status"] == 0
        T = it["T"].astype(np.float64)
        Wo, lo, io = O.cpd(T, it["R"], O.Options(seed=2 + b, compress=False, tol=TOL))
        out.append(judge(T, it["R"], *res[b], Wo, lo, 1e-6))
    summarize(out, 0.6)


def _oracle_item(args):
    import oracle as Ow
    T, R, seed, tol = args
    T = T.astype(np.float64)
    Wo, lo, _ = Ow.cpd(T, R, Ow.Options(seed=int(seed), tol=tol))
    return Wo, lo


def test_batch_full_4096_sampled_parity(cpd):
    """The uneven-batch workload: 4096 FP32 tensors, modes U{8..48}, ranks U{2..8},
    noise 1e-6; every item solved on the GPU, a seeded sample of 1024 items
    solved by the oracle (a pool of spawned processes) and held to the bar."""
    import multiprocessing as mp
    items = synth.c4_batch()
    pick = np.random.default_rng(99).choice(len(items), size=1024, replace=False)
    with mp.get_context("spawn").Pool(min(16, os.cpu_count() or 1)) as pool:
        ref = pool.map(_oracle_item, [(items[b]["T"], items[b]["R"], int(b), TOL) for b in pick], chunksize=8)
    res, infos = run_batch(cpd, items, seed=0, tol=TOL)
    assert all(inf["status"] == 0 for inf in infos)
    assert all(1 <= inf["stop"] <= 8 for inf in infos)
    out = [judge(items[int(b)]["T"].astype(np.float64), items[int(b)]["R"], *res[int(b)], Wo, lo, 1e-6)
           for b, (Wo, lo) in zip(pick, ref)]
    print({k: out.count(k) for k in ("both", "oracle_only", "gpu_only", None)})
    summarize(out, 0.75, slack=0)


def test_batch_graph_replay_and_cta_sizes(cpd):
    """On a non-default stream the batch is captured once into a CUDA graph and
    replayed: repeated calls give identical results.  Every CTA size the
    autotuner chooses between (64, 128, 256 threads, with their Gram tiles)
    solves the items to the same fits, apart from rare trajectory splits
    (an item that stalls under one Gram summation order only)."""
    items = synth.c4_batch(seed=10, B=64, lo=6, hi=30, rlo=1, rhi=6, eta=1e-6)
    Tp, offs = pack(items)
    dims = [list(it["T"].shape) for it in items]
    ranks = [it["R"] for it in items]
    st = torch.cuda.Stream()
    outs = []
    for _ in range(3):
        with torch.cuda.stream(st):
            W, lam, w_off, l_off, infos = cpd.cpd_batch_solve(Tp, offs, dims, ranks,
                                                              cpd.cpd_default_options(seed=5, tol=TOL), stream=st)
        torch.cuda.synchronize()
        outs.append((W.clone(), lam.clone()))
    assert all(torch.equal(outs[0][0], o[0]) and torch.equal(outs[0][1], o[1]) for o in outs[1:])
    fits = {}
    for th in (64, 128, 256):
        res, inf = run_batch(cpd, items, seed=5, block_threads=th, tol=TOL)
        assert all(i["status"] == 0 for i in inf)
        fits[th] = [O.fit(it["T"].astype(np.float64), *res[b]) for b, it in enumerate(items)]
    split = 0
    for b in range(len(items)):
        f = [fits[th][b] for th in (64, 128, 256)]
        if max(f) < 1e-5:
            assert max(f) - min(f) <= 1e-6, f
        elif min(f) < 1e-5:
            split += 1  # one Gram summation order stalls where another converges
    assert split <= 0.1 * len(items), split
