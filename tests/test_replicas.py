"""Multi-process path of bench.py on CPU (gloo, world size 2).

Ranks are independent replicas: the only exchange is the max of the step
time over ranks, and the whole-job rate counts every rank's units."""

import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, times, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, w, lr = bench.dist_info()
        m = bench.max_over_ranks(times[rank], w)
        out.put((r, w, lr, m, bench.whole_job_rate(1000, w, m)))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_whole_job_rate_gloo():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    times = [12.5, 40.0]
    port = _free_port()
    ps = [ctx.Process(target=_rank, args=(r, 2, port, times, q)) for r in range(2)]
    for p in ps:
        p.start()
    res = sorted(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [x[:3] for x in res] == [(0, 2, 0), (1, 2, 1)]
    assert all(x[3] == 40.0 for x in res)                  # the slowest rank's time
    assert all(abs(x[4] - 2 * 1000 / 0.040) < 1e-6 for x in res)


def test_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.0, 1) == 3.0
    assert bench.whole_job_rate(10, 1, 1000.0) == 10.0
