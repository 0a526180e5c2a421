"""Bounded device waits: a budget of one SM clock cycle makes the pipeline
waits of the tensor-core kernels (the BF16 Gram and the refinement pass) run
out at their first poll.  The call must end with CPD_ERR_TIMEOUT (not a hang,
not a NaN reported as CPD_ERR_NUMERIC), the kernels must have drained their
copies and MMAs and freed their tensor memory, and the next call with the
default budget must solve the same problem to the oracle's fit."""
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


@pytest.mark.parametrize("gram", ["fp32", "bf16"])
def test_expired_wait_reports_timeout_and_the_gpu_stays_usable(cpd, gram):
    T, _ = synth.planted(31, (64, 40, 30), 5, 0.0, 1e-4, np.float32)
    Td = torch.from_numpy(synth.flat(T)).cuda()
    bad = cpd.cpd_default_options(gram_precision=gram, refine_maxiter=3, timeout_cycles=1)
    W, lam, info, _ = cpd.cpd_dgn_solve(Td, T.shape, 5, bad)
    torch.cuda.synchronize()
    assert info["status"] == -5, info                 # CPD_ERR_TIMEOUT
    good = cpd.cpd_default_options(gram_precision=gram, refine_maxiter=3)
    W, lam, info, _ = cpd.cpd_dgn_solve(Td, T.shape, 5, good)
    torch.cuda.synchronize()
    assert info["status"] == 0, info
    T64 = T.astype(np.float64)
    Wo, lo, _ = O.cpd(T64, 5, O.Options(refine_maxiter=3))
    fg = O.fit(T64, [w.double().cpu().numpy() for w in W], lam.double().cpu().numpy())
    assert abs(fg - O.fit(T64, Wo, lo)) <= 1e-6
