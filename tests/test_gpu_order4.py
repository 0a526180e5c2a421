"""Full-size parity of the large order-4 workload: a 100x100x100x100 FP32
tensor (400 MB) of rank 15 with Gaussian factors and noise 1e-5, BF16
tensor-core compression of the first mode, dGN on the <= 15^4 core, and FP32
refinement on the full tensor, against the FP64 oracle on the same input.

The start is random (the same SplitMix64 Box-Muller draws on both sides,
Sec. 4.1.2): on this order-4, rank-15 problem the MLSVD-energy start stalls
in a local minimum (relative error ~0.3-0.46) on both sides.  The FP64 oracle
reaches the noise floor from random seeds 0, 1, 2 and 4 of 0..7; on 3, 5, 6 it
stalls and on 7 it diverges (its damping parameter falls to ~1e-55).  Seeds
0, 1 and 2 are checked: an FP32 emulation of the solver with relative
perturbations of 2e-7 on the gradient (the size of run-to-run rounding
differences) reaches the noise floor from them in 6 of 6 runs each, while from
seed 4 the trajectory passes a point (relative error ~0.4, damping at its
floor) where such perturbations decide between convergence and a stall (4 of
6), so seed 4 carries no parity claim for an FP32 solver.  The damping floor
(cpd_options.mu_min) keeps the FP32 CG well conditioned; without it seeds 1,
2 and 3 overflowed to NaN on the GPU."""
import time

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


@pytest.mark.parametrize("gram,seed", [("bf16", 0), ("bf16", 1), ("bf16", 2), ("fp32", 0)])
def test_order4_full_size_matches_oracle(cpd, gram, seed):
    c = synth.c3_order4()
    T, R = c["T"], c["R"]
    Td = torch.from_numpy(synth.flat(T)).cuda()
    opts = cpd.cpd_default_options(init="random", gram_precision=gram, refine_maxiter=20, seed=seed)
    W, lam, info, _ = cpd.cpd_dgn_solve(Td, T.shape, R, opts)            # warm-up (graph capture)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    W, lam, info, _ = cpd.cpd_dgn_solve(Td, T.shape, R, opts)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    assert info["status"] == 0
    del Td
    T64 = T.astype(np.float64)
    Wg = [w.double().cpu().numpy() for w in W]
    lg = lam.double().cpu().numpy()
    Wo, lo, io = O.cpd(T64, R, O.Options(init="random", refine_maxiter=20, seed=seed))
    fg, fo = O.fit(T64, Wg, lg), O.fit(T64, Wo, lo)
    print(f"order-4 {gram} seed {seed}: GPU solve {dt * 1e3:.1f} ms, core {info['core_dims']}, "
          f"iters {info['iters']}, refine {info['refine_iters']}; fit GPU {fg:.9e} oracle {fo:.9e}")
    assert fo < 2e-5                              # the oracle reaches the noise floor
    assert abs(fg - fo) <= 1e-6, (fg, fo, info)
    cmp = O.compare_cpd(Wg, lg, Wo, lo)
    assert max(cmp["mode_err"]) <= 1e-4 and cmp["lam_err"] <= 1e-4, cmp


def test_order4_stalled_starts_end_finite(cpd):
    """Starts on which the FP64 oracle stalls (seed 5, and the MLSVD-energy
    start) end with a normal stop and finite factors on the GPU, not with an
    overflow.  (The refinement that follows a stalled core solve continues
    with the core stage's small damping parameter and can move far from the
    stalled point; no bound on that error is claimed.)"""
    c = synth.c3_order4()
    T, R = c["T"], c["R"]
    Td = torch.from_numpy(synth.flat(T)).cuda()
    for init, seed in (("random", 5), ("mlsvd", 0)):
        opts = cpd.cpd_default_options(init=init, gram_precision="bf16", refine_maxiter=20, seed=seed)
        W, lam, info, _ = cpd.cpd_dgn_solve(Td, T.shape, R, opts)
        torch.cuda.synchronize()
        assert info["status"] == 0 and 1 <= info["stop"] <= 8, info
        assert all(bool(torch.isfinite(w).all()) for w in W) and bool(torch.isfinite(lam).all())
