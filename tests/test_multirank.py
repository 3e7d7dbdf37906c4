"""The multi-rank path of bench.py on the CPU (gloo, world size 2): every rank runs its own replica,
the timed region's time is the maximum over ranks, and the job value counts every rank's updates
(weak scaling).  No GPU and no collective on the data path."""
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = 100.0 + 50.0 * rank                    # rank 1 is the slower one
    slowest = bench._max_over_ranks(ms, dist, "cpu")
    out.put((rank, slowest, bench._job_value(world, 1_000_000, 10, slowest)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_report_the_slowest_time_and_the_whole_job_value():
    mp = pytest.importorskip("torch.multiprocessing")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [150.0, 150.0]
    # 2 replicas x 1e6 updates x 10 steps in 0.15 s
    assert all(abs(r[2] - 2 * 1e6 * 10 / 0.15 / 1e9) < 1e-12 for r in res)
