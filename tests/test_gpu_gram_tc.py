"""GPU parity of the BF16 tensor-core Gram of the first-mode unfolding.

The kernel rounds T to BF16 (round to nearest even) and accumulates in FP32,
so it is compared with the definition G = T_(1) T_(1)^T evaluated in FP64 on
the same BF16-rounded entries (tolerance: FP32 accumulation, 2e-5 of max|G|),
and with the FP64 Gram of the unrounded tensor (tolerance: BF16 input
rounding, 1e-2 of max|G|).  Shapes cover one and two 128-row tiles, N not a
multiple of 128, a ragged last 64-column step, a tensor shorter than one
step, I = 1 and the largest supported I = 256, scalar (I % 4 != 0) and
vector atomics, and both single-CTA and 8-CTA-cluster reductions (16 or more
64-column steps).  The compressed solve with BF16 compression and FP32
refinement in the original space is held to the oracle's FP64 fit.
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


def bf16_round(x):
    """FP32 -> BF16 -> FP32 with round to nearest even (finite inputs)."""
    u = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return u.astype(np.uint32).view(np.float32)


@pytest.mark.parametrize("dims", [(200, 200, 200), (128, 33, 7), (130, 5, 13), (1, 64, 2), (7, 3, 3),
                                  (256, 64, 3), (97, 11, 12), (100, 40, 30), (131, 30, 40), (256, 50, 70)])
def test_gram_bf16_matches_definition(cpd, dims):
    g = np.random.default_rng(sum(dims) + 1)
    T = g.standard_normal(dims).astype(np.float32)
    if dims == (200, 200, 200):
        T = T + 3.0                       # a dominant direction, as in a low-rank tensor
    Tf = torch.from_numpy(synth.flat(T)).cuda()
    G = cpd.cpd_mode_gram(Tf, dims, 0, precision="bf16").double().cpu().numpy()
    X = O.unfold(T.astype(np.float64), 0)
    Xb = O.unfold(bf16_round(T).astype(np.float64), 0)
    ref_b = Xb @ Xb.T
    ref = X @ X.T
    scale = np.abs(ref_b).max()
    assert np.abs(G - ref_b).max() <= 2e-5 * scale, np.abs(G - ref_b).max() / scale
    assert np.abs(G - ref).max() <= 1e-2 * scale
    # the two triangles are summed in different orders: symmetric to rounding
    assert np.abs(G - G.T).max() <= 1e-6 * scale


def test_gram_bf16_unsupported_shapes(cpd):
    T = torch.zeros(257 * 4 * 4 + 1, dtype=torch.float32, device="cuda")
    with pytest.raises(cpd.CpdError):
        cpd.cpd_mode_gram(T[:257 * 16], (257, 4, 4), 0, precision="bf16")
    with pytest.raises(cpd.CpdError):                 # not 16-byte aligned
        cpd.cpd_mode_gram(T[1:1 + 64 * 16], (64, 4, 4), 0, precision="bf16")
    with pytest.raises(cpd.CpdError):                 # modes other than the first
        cpd.cpd_mode_gram(T[:64 * 16], (64, 4, 4), 1, precision="bf16")


@pytest.mark.parametrize("seed,dims,R,rho,eta", [(142, (50, 45, 40), 5, 0.5, 1e-4),
                                                  (11, (120, 100, 90), 6, 0.5, 1e-4)])
def test_bf16_compressed_refined_solve_matches_oracle(cpd, seed, dims, R, rho, eta):
    T, Wt = synth.planted(seed, dims, R, rho, eta, np.float32)
    opts = cpd.cpd_default_options(gram_precision="bf16", refine_maxiter=20)
    W, lam, info, _ = cpd.cpd_dgn_solve(torch.from_numpy(synth.flat(T)).cuda(), T.shape, R, opts)
    torch.cuda.synchronize()
    assert info["status"] == 0
    Wg = [w.double().cpu().numpy() for w in W]
    lg = lam.double().cpu().numpy()
    T64 = T.astype(np.float64)
    Wo, lo, io = O.cpd(T64, R, O.Options(refine_maxiter=20))
    fg, fo = O.fit(T64, Wg, lg), O.fit(T64, Wo, lo)
    assert abs(fg - fo) <= 1e-6, (fg, fo, info)
    c = O.compare_cpd(Wg, lg, Wo, lo)
    assert max(c["mode_err"]) <= 1e-4 and c["lam_err"] <= 1e-4, c


def test_bf16_full_size_workload_matches_oracle(cpd):
    """The 200^3, R = 10, rho = 0.5, noise 1e-4 workload with BF16 compression
    and 20 refinement iterations, against the FP64 oracle on the same input."""
    c = synth.c2_compressed()
    T, R = c["T"], c["R"]
    opts = cpd.cpd_default_options(gram_precision="bf16", refine_maxiter=20)
    W, lam, info, _ = cpd.cpd_dgn_solve(torch.from_numpy(synth.flat(T)).cuda(), T.shape, R, opts)
    torch.cuda.synchronize()
    assert info["status"] == 0
    Wg = [w.double().cpu().numpy() for w in W]
    lg = lam.double().cpu().numpy()
    T64 = T.astype(np.float64)
    Wo, lo, io = O.cpd(T64, R, O.Options(refine_maxiter=20))
    fg, fo = O.fit(T64, Wg, lg), O.fit(T64, Wo, lo)
    assert abs(fg - fo) <= 1e-6, (fg, fo, info)
    c = O.compare_cpd(Wg, lg, Wo, lo)
    assert max(c["mode_err"]) <= 1e-4 and c["lam_err"] <= 1e-4, c
