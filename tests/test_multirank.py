"""The N > 1 path of bench.py on CPU ranks (gloo, world size 2): every rank
solves its own problem (no data-path collective); the timed region ends with
a barrier and an all-reduce MAX, and the whole-job value divides all ranks'
units by the slowest rank's time.  The reference arm runs on rank 0 only."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist            # noqa: E402
import torch.multiprocessing as mp          # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        local_ms = [120.0, 80.0][rank]                  # rank 0 is the slow one
        ms = bench.max_over_ranks(local_ms, world, "cpu")
        bench.start_barrier(world)
        val = bench.whole_job_value(1, 10, world, ms)
        out[rank] = (ms, val)
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_whole_job_value_gloo():
    world, port = 2, _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank_main, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert res[0] == res[1]                            # every rank sees the same maximum
    ms, val = res[0]
    assert ms == 120.0
    assert abs(val - 2 * 10 / 0.120) < 1e-9            # 2 ranks x 10 CPDs over the slowest 120 ms


def test_single_rank_is_unchanged():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(42.0, 1) == 42.0
    assert abs(bench.whole_job_value(4096, 3, 1, 30.0) - 4096 * 3 / 0.030) < 1e-6


def test_reference_arm_other_ranks_do_no_work():
    sys.path.insert(0, ROOT)
    import bench

    class A:
        steps, warmup, gpus = 1, 0, 2
    assert bench.run_reference(A(), rank=1, world=2) == 0
