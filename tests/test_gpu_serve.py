"""The serving loop (beagle_serve_*) on the GPU: requests from many threads, admitted under a
device-memory budget into the running persistent kernel's work queue, return the same bits as
each population scored on its own; a small request that arrives while a large one runs is
scored between the large one's work items and finishes first; oversize requests fail alone;
waits time out cleanly; the kernel is launched again after it goes idle; programs deeper than
its stack are scored too."""
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
    assert st["launches"] >= 1
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


def _c5_like(rng, P, N, d=3, lmin=40, lmax=160):
    X = rng.uniform(-3, 3, (d, N)).astype(np.float32)
    y = (np.sin(X[0]) * X[1] + X[-1]).astype(np.float32)
    return S.gen_programs(rng, P, lmin, lmax, d), X, y


def test_small_request_overtakes_a_large_one():
    """Continuous batching on the device: a small request submitted while a large one is being
    scored is admitted into the running kernel, its work interleaves with the large one's on the
    device (its %globaltimer span lies inside the large one's) and it finishes first."""
    rng = np.random.default_rng(31)
    big, Xb, yb = _c5_like(rng, 60_000, 65_536)          # ~0.1-0.2 s of device work
    small, Xs, ys = _c5_like(rng, 500, 1024, lmin=8, lmax=32)
    dsb, dss = beagle.Dataset(Xb, yb), beagle.Dataset(Xs, ys)
    srv = beagle.Server()
    import time
    tb = srv.submit(big, dsb)
    time.sleep(0.02)
    ts = srv.submit(small, dss)
    out_s = srv.wait(ts, timeout_us=60_000_000)
    done_big_when_small = srv.poll(tb)
    out_b = srv.wait(tb, timeout_us=60_000_000) if done_big_when_small is None else \
        done_big_when_small
    a, b = srv.timing(ts), srv.timing(tb)
    st = srv.stats()
    srv.destroy()
    assert done_big_when_small is None, "the large request finished before the small one"
    assert b["gpu_start_ns"] < a["gpu_start_ns"] < a["gpu_end_ns"] < b["gpu_end_ns"], (a, b)
    assert a["latency_us"] < b["latency_us"]
    assert st["launches"] == 1           # both in the same running kernel
    _same(out_s, _alone(small, dss, "fp32c"))
    _same(out_b, _alone(big, dsb, "fp32c"))
    dsb.release()
    dss.release()


def test_kernel_is_launched_again_after_it_goes_idle():
    import time
    rng = np.random.default_rng(32)
    progs, X, y = _c5_like(rng, 2000, 3000)
    ds = beagle.Dataset(X, y)
    srv = beagle.Server()
    out1 = srv.wait(srv.submit(progs, ds), timeout_us=60_000_000)
    time.sleep(0.2)                       # the kernel is stopped once no work is left
    out2 = srv.wait(srv.submit(progs, ds), timeout_us=60_000_000)
    st = srv.stats()
    srv.destroy()
    ref = _alone(progs, ds, "fp32c")
    _same(out1, ref)
    _same(out2, ref)
    assert st["launches"] == 2 and st["completed"] == 2
    ds.release()


def test_deep_programs_are_served():
    """Programs deeper than the serving kernel's 16-value stack: the kernel lists them, the
    server stops it and scores them with the 32-value deep pass; same bits as beagle_score."""
    rng = np.random.default_rng(33)
    d, N = 2, 1500
    X = rng.uniform(-1, 1, (d, N)).astype(np.float32)
    y = (X[0] * X[1]).astype(np.float32)
    progs = S.gen_programs(rng, 400, 30, 160, d, depth_cap=32, weights=(0.55, 0.1, 0.35))
    depth = np.array([S.max_depth(progs.program(p)[0]) for p in range(progs.P)])
    assert (depth > 16).any() and (depth <= 16).any()
    ds = beagle.Dataset(X, y)
    srv = beagle.Server()
    shallow = progs.subset(np.nonzero(depth <= 16)[0])
    t1 = srv.submit(progs, ds)
    t2 = srv.submit(shallow, ds)
    o1 = srv.wait(t1, timeout_us=60_000_000)
    o2 = srv.wait(t2, timeout_us=60_000_000)
    srv.destroy()
    _same(o1, _alone(progs, ds, "fp32c"))
    _same(o2, _alone(shallow, ds, "fp32c"))
    assert not np.any(beagle.unpack_fitness(o1)[2] & beagle.FLAG_MALFORMED)
    ds.release()
