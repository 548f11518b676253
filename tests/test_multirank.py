"""Host logic of the multi-rank benchmark path on CPU (gloo, world size 2).

Each rank runs the whole path on its own frame (independent problems, no
data-path collective); the only cross-rank step is the max of the per-rank
timed regions. These tests run that step over gloo with two processes and
check the whole-job aggregation and that only rank 0 reports.
"""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as tdist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import sys
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    tdist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        # rank r "took" 10 + r ms for the device region and 20 - r for end to end
        got = bench.reduce_max_over_ranks([10.0 + rank, 20.0 - rank])
        ref = bench.run_reference(type("A", (), {"steps": 1, "warmup": 0})(), rank, world) \
            if rank == 1 else "skipped"
        out[rank] = (got, ref)
    finally:
        tdist.destroy_process_group()


def test_max_over_ranks_and_rank0_only_reporting():
    world = 2
    port = _free_port()
    with mp.get_context("spawn").Manager() as m:  # no fork of a process that may run OpenMP threads
        out = m.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for r in range(world):
        assert res[r][0] == [11.0, 20.0]
    assert res[1][1] is None  # the reference arm prints nothing off rank 0


def test_whole_job_rate():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    # 2 ranks x 5 steps x 1000 windows in 10 ms (slowest rank) = 1e6 windows/s
    assert bench.whole_job_rate(1000, 5, 2, 10.0) == pytest.approx(1.0e6)
    assert bench.windows_per_step(1024, 1024) == 8602224
