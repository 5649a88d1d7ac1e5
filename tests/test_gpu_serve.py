"""The serving loop (beagle_serve_*) on the GPU: requests from many threads, admitted under a
device-memory budget and packed into shared launches, return the same bits as each population
scored on its own; oversize requests fail alone; waits time out cleanly."""
from __future__ import annotations

import threading

import numpy as np
import pytest

from paper_2607_06731_gb300 import beagle, synth as S
from tests import parity

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    yield


def _runs(n_runs=4, seed=21):
    """Independent evolutionary runs: each its own dataset and a few generations."""
    rng = np.random.default_rng(seed)
    runs = []
    for r in range(n_runs):
        d = int(rng.integers(1, 6))
        N = int(rng.integers(100, 3000))
        X = rng.uniform(-1, 1, (d, N)).astype(np.float32)      # column-major [d][N]
        y = (np.sin(X[0]) + X[-1] ** 2).astype(np.float32)
        ds = beagle.Dataset(X, y)
        gens = []
        for g in range(3):
            P = int(rng.integers(1, 700))
            gens.append(S.gen_programs(rng, P, 1, int(rng.integers(8, 80)), d))
        runs.append((X, y, ds, gens))
    return runs


def _alone(progs, ds, precision):
    dp = beagle.DevicePrograms(progs)
    out = beagle.score_programs(dp, ds, precision=precision)
    torch.cuda.synchronize()
    return beagle.unpack_fitness(out)


def _same(got, ref):
    for a, b in zip(beagle.unpack_fitness(got), ref):
        assert np.array_equal(a, b, equal_nan=True)


@pytest.mark.parametrize("precision", ["fp32c", "fp64"])
def test_concurrent_requests_equal_alone(precision):
    runs = _runs()
    refs = [[_alone(p, ds, precision) for p in gens] for _, _, ds, gens in runs]
    srv = beagle.Server(max_inflight=3, max_batch_jobs=5, precision=precision)
    results = {}
    errors = []

    def client(i):
        try:
            _, _, ds, gens = runs[i]
            for g, p in enumerate(gens):     # one generation at a time, like an EA loop
                t = srv.submit(p, ds)
                results[(i, g)] = srv.wait(t, timeout_us=60_000_000)
        except Exception as e:   # surfaced below
            errors.append(e)

    th = [threading.Thread(target=client, args=(i,)) for i in range(len(runs))]
    for t in th:
        t.start()
    for t in th:
        t.join()
    assert not errors, errors
    for i, (_, _, _, gens) in enumerate(runs):
        for g in range(len(gens)):
            _same(results[(i, g)], refs[i][g])
    st = srv.stats()
    n = sum(len(g) for *_, g in runs)
    assert st["submitted"] == n and st["completed"] == n and st["rejected"] == 0
    assert st["queued"] == 0 and st["bytes_in_use"] == 0
    evals = sum(int(p.lengths.sum()) * X.shape[1] for X, _, _, gens in runs for p in gens)
    assert st["node_evals"] == evals
    assert 0 < st["p50_us"] <= st["p99_us"] <= st["max_us"]
    assert st["peak_bytes"] <= st["budget_bytes"]
    srv.destroy()
    for *_, ds, _ in runs:
        ds.release()


def test_budget_limits_device_bytes_and_queues_the_rest():
    runs = _runs(n_runs=3, seed=5)
    reqs = [(ds, p) for _, _, ds, gens in runs for p in gens]
    # room for about two requests at a time
    sizes = []
    for ds, p in reqs:
        tiles = (ds.N + 511) // 512
        sizes.append(p.lengths.size * (44 * tiles + 24 + 12 + 4) + 5 * int(p.lengths.sum()))
    budget = 2 * max(sizes) + (1 << 16)
    srv = beagle.Server(hbm_budget_bytes=budget, max_inflight=4, max_batch_jobs=64)
    tickets = [srv.submit(p, ds) for ds, p in reqs]
    outs = [srv.wait(t, timeout_us=60_000_000) for t in tickets]
    st = srv.stats()
    assert st["completed"] == len(reqs)
    assert 0 < st["peak_bytes"] <= budget
    assert st["launches"] >= 2
    for (ds, p), o in zip(reqs, outs):
        _same(o, _alone(p, ds, "fp32c"))
    srv.destroy()
    for *_, ds, _ in runs:
        ds.release()


def test_oversize_request_fails_alone():
    rng = np.random.default_rng(3)
    X = rng.uniform(-1, 1, (2, 4096)).astype(np.float32)
    y = (X[0] * X[1]).astype(np.float32)
    ds = beagle.Dataset(X, y)
    small = S.gen_programs(rng, 10, 1, 12, 2)
    big = S.gen_programs(rng, 20000, 1, 12, 2)
    srv = beagle.Server(hbm_budget_bytes=200_000, max_inflight=2)
    t1 = srv.submit(small, ds)
    t2 = srv.submit(big, ds)
    t3 = srv.submit(small, ds)
    a = srv.wait(t1, timeout_us=30_000_000)
    with pytest.raises(beagle.BeagleError) as ei:
        srv.wait(t2, timeout_us=30_000_000)
    assert ei.value.code == beagle.ERR_OOM
    c = srv.wait(t3, timeout_us=30_000_000)
    _same(a, _alone(small, ds, "fp32c"))
    _same(c, _alone(small, ds, "fp32c"))
    assert srv.stats()["rejected"] == 1
    srv.destroy()
    ds.release()


def test_wait_timeout_keeps_the_ticket_and_poll_collects():
    pr = S.make_c2(seed=2, P=20_000)           # a few ms of work
    ds = beagle.Dataset(pr.X, pr.y)
    srv = beagle.Server()
    t = srv.submit(pr.programs, ds)
    out = None
    try:
        out = srv.wait(t, timeout_us=0)
    except beagle.BeagleError as e:
        assert e.code == beagle.ERR_TIMEOUT
    while out is None:
        out = srv.poll(t)
    ref = _alone(pr.programs, ds, "fp32c")
    _same(out, ref)
    with pytest.raises(beagle.BeagleError):
        srv.poll(t)                              # retired
    srv.destroy()
    ds.release()


def test_served_results_match_the_oracle_on_a_sample():
    runs = _runs(n_runs=2, seed=8)
    srv = beagle.Server()
    for k, (X, y, ds, gens) in enumerate(runs):
        p = gens[0]
        got = srv.wait(srv.submit(p, ds))
        idx = np.sort(np.random.default_rng(k).choice(len(p.lengths), min(len(p.lengths), 400),
                                                      replace=False))
        refs = parity.references(p.subset(idx), X, y)
        parity.check_fp32(tuple(a[idx] for a in beagle.unpack_fitness(got)), refs,
                          name=f"serve-{k}")
    srv.destroy()
    for *_, ds, _ in runs:
        ds.release()
