"""beagle_score_static: scoring with the library's fixed scratch array instead of allocated
device memory, for callers that cannot allocate while they score (a loop that must not block
on a device synchronisation, a process with a fixed up-front memory budget). Its results
must match beagle_score's on consecutive calls; this file runs last (it is collected last)."""
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


def _static_call(dp, ds, out, precision):
    return beagle.lib().beagle_score_static(
        dp.ops.data_ptr(), dp.offsets.data_ptr(), dp.lengths.data_ptr(), dp.consts.data_ptr(),
        dp.P, ds.id, out.data_ptr(), precision, torch.cuda.current_stream().cuda_stream)


def test_static_scratch_matches_score_on_consecutive_calls():
    rng = np.random.default_rng(8)
    X2 = rng.uniform(-3, 3, size=(3, 2500)).astype(np.float32)
    y2 = (X2[0] * X2[1] + np.sin(X2[2])).astype(np.float32)
    workloads = [S.make_c1(), S.Problem("multi-tile", S.gen_programs(rng, 900, 4, 64, 3), X2, y2, {})]
    for prec in (beagle.FP32_COMPENSATED, beagle.FP64):
        for pr in workloads:          # two calls in a row on different workloads
            ds = beagle.Dataset(pr.X, pr.y)
            dp = beagle.DevicePrograms(pr.programs)
            ref = beagle.unpack_fitness(beagle.score_programs(dp, ds, precision=prec))
            out = torch.full((dp.P, 3), float("nan"), dtype=torch.float64, device="cuda")
            beagle.check(_static_call(dp, ds, out, prec))
            torch.cuda.synchronize()
            got = beagle.unpack_fitness(out)
            tol = parity.TOL32 if prec == beagle.FP32_COMPENSATED else parity.TOL64
            assert np.array_equal(got[2], ref[2])
            assert np.all(parity.close(got[0], ref[0], *tol))
            assert np.all(parity.close(got[1], ref[1], *tol))
            ds.release()


def test_static_scratch_rejects_requests_above_its_limit():
    pr = S.make_c1(P=64)
    ds = beagle.Dataset(pr.X, pr.y)
    dp = beagle.DevicePrograms(pr.programs)
    out = torch.empty((dp.P, 3), dtype=torch.float64, device="cuda")
    # 10^6 programs x 1 tile x 44 bytes > 32 MiB: refused before any device work is enqueued.
    rc = beagle.lib().beagle_score_static(
        dp.ops.data_ptr(), dp.offsets.data_ptr(), dp.lengths.data_ptr(), dp.consts.data_ptr(),
        1_000_000, ds.id, out.data_ptr(), beagle.FP32_COMPENSATED,
        torch.cuda.current_stream().cuda_stream)
    assert rc == -8 and "limit" in beagle.last_error()
    ds.release()
