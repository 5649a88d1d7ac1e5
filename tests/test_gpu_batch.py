"""Ragged batches, graph-captured plans and the autotuner (GPU)."""
from __future__ import annotations

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


def _ragged(n=10, scale=0.01, seed=4):
    pops = S.make_c4(seed=seed, n_pops=n, scale=scale)
    items = []
    for pr in pops:
        ds = beagle.Dataset(pr.X, pr.y)
        dp = beagle.DevicePrograms(pr.programs)
        out = torch.full((dp.P, 3), float("nan"), dtype=torch.float64, device="cuda")
        items.append((dp, ds, out))
    return pops, items


def _alone(items, precision="fp32c"):
    res = []
    for dp, ds, _ in items:
        res.append(beagle.unpack_fitness(beagle.score_programs(dp, ds, precision=precision)))
    torch.cuda.synchronize()
    return res


def test_batch_equals_jobs_scored_alone():
    """Ragged populations (P, L, N, d all differ) in one launch give the same bits as each
    population scored on its own."""
    pops, items = _ragged()
    for prec in ("fp32c", "fp64"):
        ref = _alone(items, prec)
        beagle.score_batch(items, precision=prec)
        torch.cuda.synchronize()
        for (dp, ds, out), r in zip(items, ref):
            got = beagle.unpack_fitness(out)
            for a, b in zip(got, r):
                assert np.array_equal(a, b, equal_nan=True)
    for _, ds, _ in items:
        ds.release()


def test_batch_matches_oracle_on_a_sample():
    pops, items = _ragged(n=6, scale=0.02, seed=9)
    beagle.score_batch(items)
    torch.cuda.synchronize()
    rng = np.random.default_rng(0)
    for k, (pr, (dp, ds, out)) in enumerate(zip(pops, items)):
        got = beagle.unpack_fitness(out)
        idx = rng.choice(pr.programs.P, min(400, pr.programs.P), replace=False)
        refs = parity.references(pr.programs.subset(idx), pr.X, pr.y)
        parity.check_fp32(tuple(a[idx] for a in got), refs, name=f"batch-{k}")
        ds.release()


def test_graph_plan_replays_the_batch():
    pops, items = _ragged(n=5, scale=0.01, seed=11)
    ref = _alone(items)
    plan = beagle.BatchPlan(items)
    with pytest.raises(beagle.BeagleError):
        items[0][1].release()                  # held by the plan
    for _ in range(3):
        for _, _, out in items:
            out.fill_(float("nan"))
        plan.launch()
        torch.cuda.synchronize()
        for (dp, ds, out), r in zip(items, ref):
            got = beagle.unpack_fitness(out)
            for a, b in zip(got, r):
                assert np.array_equal(a, b, equal_nan=True)
    plan.destroy()
    for _, ds, _ in items:
        ds.release()


def test_autotuner_picks_a_shape_and_results_stay_in_tolerance():
    pops, items = _ragged(n=4, scale=0.01, seed=13)
    ref = _alone(items)
    cfg, ms = beagle.autotune(items, max_trials=6)
    assert cfg["cases_per_lane"] in (2, 4, 8) and cfg["tile"] in (256, 512) and ms > 0
    after = _alone(items)                      # now uses the tuned shape for this class
    for r, a in zip(ref, after):
        assert np.array_equal(r[2], a[2])
        assert np.all(parity.close(a[0], r[0], 1e-6, 1e-9))
        assert np.all(parity.close(a[1], r[1], 1e-6, 1e-9))
    beagle.autotune_clear()
    for _, ds, _ in items:
        ds.release()


def test_launch_configurations_agree():
    """Every cases-per-lane variant gives the same bits at a fixed tile."""
    pr = S.make_c2(P=2000)
    ds = beagle.Dataset(pr.X, pr.y)
    dp = beagle.DevicePrograms(pr.programs)
    try:
        for tile, variants in ((512, (2, 4, 8)), (256, (2, 4, 8))):
            beagle.set_launch_config(cases_per_lane=variants[0], tile=tile)
            ref = beagle.unpack_fitness(beagle.score_programs(dp, ds))
            for cases in variants:
                for group in (0, 40):
                    beagle.set_launch_config(cases_per_lane=cases, tile=tile, group=group)
                    got = beagle.unpack_fitness(beagle.score_programs(dp, ds))
                    for a, b in zip(got, ref):
                        assert np.array_equal(a, b, equal_nan=True), (tile, cases, group)
        # the automatic shape (no launch configuration) is one of them
        beagle.reset_launch_config()
        auto = beagle.unpack_fitness(beagle.score_programs(dp, ds))
        beagle.set_launch_config(cases_per_lane=4, tile=512)
        ref = beagle.unpack_fitness(beagle.score_programs(dp, ds))
        for a, b in zip(auto, ref):
            assert np.array_equal(a, b, equal_nan=True)
    finally:
        beagle.reset_launch_config()
    ds.release()


@pytest.mark.parametrize("cases", [4, 8])
def test_stack_in_tensor_memory_at_every_warp_count(cases):
    """The 4-case kernel allocates 64 tensor-memory columns per four consumer warps (64 at one
    warp, 512 at 31), the 8-case kernel 128 (128 at one warp, 512 at 16), and each gives warp
    w the columns of slot w / 4 in lane quarter w % 4: the same bits at every warp count and
    with grids smaller or larger than the SM count."""
    pr = S.make_c2(P=1500)
    ds = beagle.Dataset(pr.X, pr.y)
    dp = beagle.DevicePrograms(pr.programs)
    try:
        beagle.set_launch_config(cases_per_lane=4, tile=512)
        ref = beagle.unpack_fitness(beagle.score_programs(dp, ds))
        for warps, grid in ((1, 0), (3, 0), (4, 0), (5, 0), (8, 0), (13, 0), (16, 0), (31, 0),
                            (2, 7), (6, 300)):
            beagle.set_launch_config(cases_per_lane=cases, tile=512, warps=warps, grid=grid)
            got = beagle.unpack_fitness(beagle.score_programs(dp, ds))
            for a, b in zip(got, ref):
                assert np.array_equal(a, b, equal_nan=True), (warps, grid)
    finally:
        beagle.reset_launch_config()
    ds.release()


def test_plan_capture_as_the_first_call_of_a_process():
    """A graph-captured plan built before any other scoring call in a fresh process (pool
    set-up and kernel loading happen before the capture begins)."""
    import subprocess
    import sys
    import textwrap
    code = textwrap.dedent("""
        import numpy as np, torch
        from paper_2607_06731_gb300 import beagle, synth as S
        pops = S.make_c4(seed=11, n_pops=5, scale=0.01)
        items = []
        for pr in pops:
            items.append((beagle.DevicePrograms(pr.programs), beagle.Dataset(pr.X, pr.y),
                          torch.full((pr.programs.P, 3), float("nan"), dtype=torch.float64,
                                     device="cuda")))
        plan = beagle.BatchPlan(items)
        plan.launch()
        torch.cuda.synchronize()
        for dp, ds, out in items:
            ref = beagle.unpack_fitness(beagle.score_programs(dp, ds))
            got = beagle.unpack_fitness(out)
            torch.cuda.synchronize()
            assert all(np.array_equal(a, b, equal_nan=True) for a, b in zip(got, ref))
        print("ok")
    """)
    import os
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "-c", code], cwd=root, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0 and r.stdout.strip().endswith("ok"), r.stderr[-2000:]
