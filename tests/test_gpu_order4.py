"""Full-size parity of the large order-4 workload: a 100x100x100x100 FP32
tensor (400 MB) of rank 15 with Gaussian factors and noise 1e-5, BF16
tensor-core compression of the first mode, dGN on the <= 15^4 core, and FP32
refinement on the full tensor, against the FP64 oracle on the same input.

The start is random (the same SplitMix64 Box-Muller draws on both sides,
Sec. 4.1.2): on this order-4, rank-15 problem the MLSVD-energy start stalls
in a local minimum (fit ~0.2) on both sides, so the random start is the one
the method is run with here, with a seed whose start converges (with other
seeds the random start can stall too; a stalled FP32 trajectory, whose
damping parameter falls to ~1e-8, can then overflow where the FP64 oracle
only stalls)."""
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


@pytest.mark.parametrize("gram", ["bf16", "fp32"])
def test_order4_full_size_matches_oracle(cpd, gram):
    c = synth.c3_order4()
    T, R = c["T"], c["R"]
    Td = torch.from_numpy(synth.flat(T)).cuda()
    opts = cpd.cpd_default_options(init="random", gram_precision=gram, refine_maxiter=5, seed=0)
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
    Wo, lo, io = O.cpd(T64, R, O.Options(init="random", refine_maxiter=5, seed=0))
    fg, fo = O.fit(T64, Wg, lg), O.fit(T64, Wo, lo)
    print(f"order-4 {gram}: GPU solve {dt * 1e3:.1f} ms, core {info['core_dims']}, iters {info['iters']}, "
          f"refine {info['refine_iters']}; fit GPU {fg:.9e} oracle {fo:.9e}")
    assert fo < 2e-5                              # the oracle reaches the noise floor
    assert abs(fg - fo) <= 1e-6, (fg, fo, info)
    cmp = O.compare_cpd(Wg, lg, Wo, lo)
    assert max(cmp["mode_err"]) <= 1e-4 and cmp["lam_err"] <= 1e-4, cmp
