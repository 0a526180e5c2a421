"""GPU parity of the batched solver (one persistent launch, one CTA per CPD)
against the FP64 oracle run item by item with the same options and seeds.

Parity is asserted where the method itself reaches the noise floor on the
oracle's side (planted problems with the MLSVD-energy start occasionally
stall in a local minimum; those items are counted and excluded, and most
items must converge).  dGN converges to a local minimum (Sec. 3.5) and some
starts lead into one (Sec. 4.1.2): starts that agree to FP32 rounding can
end at different stationary points, so an item on which only the GPU run
stalls is a trajectory split, not a parity failure; splits must be rare
(at most 10% of the items the oracle solves) and end with a normal stop.  These workloads have noise 1e-6 = tol: the
improvement stop test (|e_{k-1} - e_k| < tol) then fires at an iteration
that depends on rounding, so FP32 and FP64 runs end a few iterations apart
and their fits differ by up to a few tol.  The bar is therefore: a large
majority of items within 1e-6 absolute of the oracle's fit (with factors
within 1e-4 after alignment), and every converged item within 5e-6."""
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


def check_item(it, Wg, lg, seed, rel_eta):
    """Returns None when the oracle stalls (not converged), "split" when only
    the GPU run stalls, else True when the GPU result meets the 1e-6 fit bar
    (factors then checked), False when it does not (but is within 5e-6)."""
    T = it["T"].astype(np.float64)
    Wo, lo, io = O.cpd(T, it["R"], O.Options(seed=int(seed)))
    fo, fg = O.fit(T, Wo, lo), O.fit(T, Wg, lg)
    if fo >= 10 * rel_eta:
        return None
    if fg >= 10 * rel_eta:
        return "split"
    assert abs(fg - fo) <= 5e-6, (fg, fo, it["T"].shape, it["R"])
    if abs(fg - fo) > 1e-6:
        return False
    c = O.compare_cpd(Wg, lg, Wo, lo)
    assert max(c["mode_err"]) <= 1e-4 and c["lam_err"] <= 1e-4, c
    return True


def summarize(results, min_converged, min_within, max_split=0.1):
    conv = [r for r in results if r is not None]
    assert len(conv) >= min_converged * len(results), (len(conv), len(results))
    split = [r for r in conv if r == "split"]
    assert len(split) <= max_split * len(conv), (len(split), len(conv))
    both = [r for r in conv if r != "split"]
    assert sum(both) >= min_within * len(both), (sum(both), len(both))


def test_batch_small_uneven_matches_oracle(cpd):
    items = synth.c4_batch(seed=7, B=48, lo=6, hi=20, rlo=1, rhi=6, eta=1e-6)
    res, infos = run_batch(cpd, items, seed=11)
    out = []
    for b, (it, (Wg, lg)) in enumerate(zip(items, res)):
        assert infos[b]["status"] == 0
        out.append(check_item(it, Wg, lg, 11 + b, 1e-6))
    summarize(out, 0.8, 0.85)


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
    res, infos = run_batch(cpd, items, seed=1)
    out = []
    for b, it in enumerate(items):
        assert infos[b]["status"] == 0
        out.append(check_item(it, *res[b], 1 + b, 1e-6))
    summarize(out, 0.6, 0.6)


def test_batch_uncompressed(cpd):
    items = synth.c4_batch(seed=9, B=8, lo=4, hi=9, rlo=1, rhi=3, eta=1e-6)
    res, infos = run_batch(cpd, items, seed=2, compress=0)
    for b, it in enumerate(items):
        T = it["T"].astype(np.float64)
        Wo, lo, io = O.cpd(T, it["R"], O.Options(seed=2 + b, compress=False))
        fo, fg = O.fit(T, Wo, lo), O.fit(T, *res[b])
        if fo < 1e-5:
            assert abs(fg - fo) <= 1e-6


def test_batch_full_4096_sampled_parity(cpd):
    """The uneven-batch workload: 4096 FP32 tensors, modes U{8..48}, ranks U{2..8},
    noise 1e-6; every item solved, a seeded sample checked against the oracle."""
    items = synth.c4_batch()
    res, infos = run_batch(cpd, items, seed=0)
    assert all(inf["status"] == 0 for inf in infos)
    assert all(1 <= inf["stop"] <= 8 for inf in infos)
    pick = np.random.default_rng(123).choice(len(items), size=32, replace=False)
    out = [check_item(items[int(b)], *res[int(b)], int(b), 1e-6) for b in pick]
    summarize(out, 0.75, 0.85)


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
            W, lam, w_off, l_off, infos = cpd.cpd_batch_solve(Tp, offs, dims, ranks, cpd.cpd_default_options(seed=5),
                                                              stream=st)
        torch.cuda.synchronize()
        outs.append((W.clone(), lam.clone()))
    assert all(torch.equal(outs[0][0], o[0]) and torch.equal(outs[0][1], o[1]) for o in outs[1:])
    fits = {}
    for th in (64, 128, 256):
        res, inf = run_batch(cpd, items, seed=5, block_threads=th)
        assert all(i["status"] == 0 for i in inf)
        fits[th] = [O.fit(it["T"].astype(np.float64), *res[b]) for b, it in enumerate(items)]
    split = 0
    for b in range(len(items)):
        f = [fits[th][b] for th in (64, 128, 256)]
        if max(f) < 1e-5:
            assert max(f) - min(f) <= 5e-6, f
        elif min(f) < 1e-5:
            split += 1  # one Gram summation order stalls where another converges
    assert split <= 0.1 * len(items), split
