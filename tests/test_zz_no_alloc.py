"""beagle_score_static: scoring with the library's fixed scratch array instead of allocated
device memory, for callers that cannot allocate while they score (a loop that must not block
on a device synchronisation, a process with a fixed up-front memory budget). Its results must
be the same bits as beagle_score's (automatic launch shape) on consecutive calls, it must
refuse sizes above its limit, and it must not allocate from the device's memory pool. This
file runs last (it is collected last)."""
from __future__ import annotations

import ctypes

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
    beagle.reset_launch_config()
    beagle.autotune_clear()
    yield


def _static_call(dp, ds, out, precision, P=None):
    return beagle.lib().beagle_score_static(
        dp.ops.data_ptr(), dp.offsets.data_ptr(), dp.lengths.data_ptr(), dp.consts.data_ptr(),
        dp.P if P is None else P, ds.id, out.data_ptr(), precision,
        torch.cuda.current_stream().cuda_stream)


def _workloads():
    rng = np.random.default_rng(8)
    X2 = rng.uniform(-3, 3, size=(3, 2500)).astype(np.float32)
    y2 = (X2[0] * X2[1] + np.sin(X2[2])).astype(np.float32)
    return [S.make_c1(), S.Problem("multi-tile", S.gen_programs(rng, 900, 4, 64, 3), X2, y2, {})]


def test_static_scratch_matches_score_on_consecutive_calls():
    for prec in (beagle.FP32_COMPENSATED, beagle.FP64):
        for pr in _workloads():          # two calls in a row on different workloads
            ds = beagle.Dataset(pr.X, pr.y)
            dp = beagle.DevicePrograms(pr.programs)
            ref = beagle.unpack_fitness(beagle.score_programs(dp, ds, precision=prec))
            out = torch.full((dp.P, 3), float("nan"), dtype=torch.float64, device="cuda")
            beagle.check(_static_call(dp, ds, out, prec))
            torch.cuda.synchronize()
            got = beagle.unpack_fitness(out)
            # same tile (512 cases), same per-program sums: the same bits
            for a, b in zip(got, ref):
                assert np.array_equal(a, b, equal_nan=True)
            ds.release()


def test_static_scratch_rejects_requests_above_its_limit():
    pr = S.make_c1(P=64)
    ds = beagle.Dataset(pr.X, pr.y)
    dp = beagle.DevicePrograms(pr.programs)
    out = torch.empty((dp.P, 3), dtype=torch.float64, device="cuda")
    # 10^6 programs x 1 tile x 44 bytes > 32 MiB, and sizes whose byte count would wrap a
    # 64-bit product: refused before any device work is enqueued.
    for P in (1_000_000, 1 << 31, 1 << 62):
        rc = _static_call(dp, ds, out, beagle.FP32_COMPENSATED, P=P)
        assert rc == -8 and ("limit" in beagle.last_error() or "2^31" in beagle.last_error())
    ds.release()


class _Pool:
    """The device's default memory pool through the driver API: the pool that stream-ordered
    allocations (cudaMallocAsync) come from."""
    USED_MEM_CURRENT, USED_MEM_HIGH = 7, 8

    def __init__(self):
        self.cu = ctypes.CDLL("libcuda.so.1")
        dev = ctypes.c_int()
        assert self.cu.cuDeviceGet(ctypes.byref(dev), torch.cuda.current_device()) == 0
        self.pool = ctypes.c_void_p()
        assert self.cu.cuDeviceGetDefaultMemPool(ctypes.byref(self.pool), dev) == 0

    def get(self, attr):
        v = ctypes.c_uint64()
        assert self.cu.cuMemPoolGetAttribute(self.pool, attr, ctypes.byref(v)) == 0
        return v.value

    def reset_high(self):
        z = ctypes.c_uint64(0)
        assert self.cu.cuMemPoolSetAttribute(self.pool, self.USED_MEM_HIGH, ctypes.byref(z)) == 0


def test_static_scratch_allocates_nothing():
    pr = _workloads()[1]
    ds = beagle.Dataset(pr.X, pr.y)
    dp = beagle.DevicePrograms(pr.programs)
    out = torch.empty((dp.P, 3), dtype=torch.float64, device="cuda")
    beagle.check(_static_call(dp, ds, out, beagle.FP32_COMPENSATED))   # first call: set-up
    torch.cuda.synchronize()
    pool = _Pool()
    torch_before = torch.cuda.memory_allocated()
    base = pool.get(pool.USED_MEM_CURRENT)
    pool.reset_high()
    for _ in range(2):
        beagle.check(_static_call(dp, ds, out, beagle.FP32_COMPENSATED))
    torch.cuda.synchronize()
    assert pool.get(pool.USED_MEM_HIGH) <= base, "beagle_score_static allocated device memory"
    assert torch.cuda.memory_allocated() == torch_before
    # the same check sees beagle_score's stream-ordered scratch
    pool.reset_high()
    beagle.score_programs(dp, ds, out=out)
    torch.cuda.synchronize()
    assert pool.get(pool.USED_MEM_HIGH) > base
    ds.release()
