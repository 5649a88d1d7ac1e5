"""The replicas-only multi-GPU path of bench.py on CPU: two gloo ranks on 127.0.0.1 agree on
the slowest rank's time, the whole-job value counts every rank's population, and the
reference arm runs on rank 0 alone."""
from __future__ import annotations

import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist          # noqa: E402
import torch.multiprocessing as mp        # noqa: E402


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mine = 10.0 + 5.0 * rank                      # rank 1 is the slow one
        slowest = bench.max_over_ranks(mine, dist, "cpu")
        r, w, lr = bench.dist_env()

        class A:
            P, steps, warmup = 1000, 1, 0
        rc = bench.run_reference(A, rank, world) if rank == 1 else 0
        out.put((rank, slowest, (r, w, lr), rc))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_the_slowest_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    assert [g[1] for g in got] == [15.0, 15.0]
    assert got[0][2] == (0, 2, 0) and got[1][2] == (1, 2, 1)
    assert got[1][3] == 0                           # the reference arm's other ranks do no work


def test_whole_job_value_counts_every_rank():
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import bench
    one = bench.whole_job_gpops(10**9, 4, 1, 2000.0)
    assert one == pytest.approx(2.0)
    assert bench.whole_job_gpops(10**9, 4, 4, 2000.0) == pytest.approx(4 * one)
    assert bench.max_over_ranks(3.5, None, "cpu") == 3.5
