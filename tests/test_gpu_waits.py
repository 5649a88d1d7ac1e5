"""Bounded device waits (GPU): when the producer warp publishes nothing (test hook), every
consumer's mbarrier wait runs out after the configured limit, the launch ends with the error
word set, every result carries FLAG_TIMEOUT, and the context stays usable for the next call.
No fault, trap or hang is involved: the waits are bounded and no copy is in flight."""
from __future__ import annotations

import time

import numpy as np
import pytest

from paper_2607_06731_gb300 import beagle, synth as S

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    yield


def test_wait_limit_reports_timeout_and_context_stays_usable(monkeypatch):
    pr = S.make_c1()
    ds = beagle.Dataset(pr.X, pr.y)
    dp = beagle.DevicePrograms(pr.programs)
    ref = beagle.unpack_fitness(beagle.score_programs(dp, ds))
    torch.cuda.synchronize()

    monkeypatch.setenv("BEAGLE_WAIT_LIMIT_US", "20000")
    monkeypatch.setenv("BEAGLE_TEST_STALL", "1")
    t0 = time.perf_counter()
    out = beagle.score_programs(dp, ds)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    mse, omr, flags = beagle.unpack_fitness(out)
    assert (flags == 8).all()                    # BEAGLE_FLAG_TIMEOUT on every program
    assert np.isnan(mse).all() and np.isnan(omr).all()
    assert dt < 5.0                              # the 20 ms limit, not the 4 s default

    monkeypatch.delenv("BEAGLE_TEST_STALL")
    again = beagle.unpack_fitness(beagle.score_programs(dp, ds))
    torch.cuda.synchronize()
    for a, b in zip(again, ref):
        assert np.array_equal(a, b, equal_nan=True)
    ds.release()
