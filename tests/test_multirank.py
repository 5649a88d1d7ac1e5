"""The multi-GPU paths on CPU, as gloo ranks on 127.0.0.1: the benchmark's replicas agree on the
slowest rank's time, the whole-job value counts every rank's population, and the reference
arm runs on rank 0 alone; a population sharded by cost over the ranks (beagle_shard_by_cost,
multigpu.score_sharded; the oracle stands in for each rank's GPU) gathers to the same
fitness as scoring it whole."""
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


def test_shard_by_cost_balances_summed_lengths():
    from paper_2607_06731_gb300 import beagle, synth as S
    import numpy as np
    rng = np.random.default_rng(1)
    lengths = rng.integers(1, 257, 100_001).astype(np.int32)
    for world in (1, 2, 3, 8, 64):
        b = beagle.shard_by_cost(lengths, world)
        assert b[0] == 0 and b[-1] == len(lengths) and np.all(np.diff(b) >= 0)
        cost = np.add.reduceat(lengths.astype(np.int64), b[:-1]) if world > 1 else [lengths.sum()]
        assert np.max(np.abs(np.asarray(cost) - lengths.sum() / world)) <= lengths.max()
    # more shards than programs: empty shards, nothing lost
    b = beagle.shard_by_cost(np.array([5, 7], np.int32), 4)
    assert b[0] == 0 and b[-1] == 2 and np.all(np.diff(b) >= 0)


def _shard_main(rank, world, port, out):
    import sys
    import numpy as np
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import oracle
    from paper_2607_06731_gb300 import multigpu, synth as S
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        pr = S.make_c2(P=900, N=256)

        def score(sub):
            m, r, f = oracle.score_programs(sub, pr.X, pr.y, "fp64", nthreads=1)
            return np.stack([m, r, f.astype(np.float64)], axis=1)
        got = multigpu.score_sharded(pr.programs, score, rank, world, dist)
        (a, b), _ = multigpu.shard(pr.programs, rank, world)
        out.put((rank, a, b, got))
    finally:
        dist.destroy_process_group()


def test_sharded_scoring_gathers_the_whole_population():
    import numpy as np
    import oracle
    from paper_2607_06731_gb300 import synth as S
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    world = 2
    procs = [ctx.Process(target=_shard_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    res.sort()
    pr = S.make_c2(P=900, N=256)
    m, r, f = oracle.score_programs(pr.programs, pr.X, pr.y, "fp64")
    whole = np.stack([m, r, f.astype(np.float64)], axis=1)
    assert res[0][1] == 0 and res[0][2] == res[1][1] and res[1][2] == pr.programs.P
    for _, _, _, got in res:                    # every rank holds the whole result
        assert np.array_equal(got, whole)
