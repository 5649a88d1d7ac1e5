"""Accuracy of the FP32 path's sin, cos, exp and protected log (GPU), through beagle_eval on
one-token programs.

The oracle's error bound takes the device's transcendentals to within 2 ulp of the exact
value (the bound CUDA documents for sinf, cosf and expf; exp is CUDA's expf); the library's own
branch-free sin, cos and log (range reduction plus fitted polynomials; CUDA's sinf/cosf above
65536) must meet it on every
argument class a program can produce: small, moderate, near multiples of pi/2 (sin, cos),
overflow and underflow (exp), the whole valid range of both signs and the 1e-3 threshold
(protected log).
"""
from __future__ import annotations

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


def _arguments(n=1 << 20, seed=12):
    rng = np.random.default_rng(seed)
    parts = [
        rng.uniform(-4, 4, n),
        rng.uniform(-200, 200, n),
        rng.uniform(-65536, 65536, n),
        np.exp(rng.uniform(np.log(1e-30), np.log(1e-2), n)) * rng.choice([-1, 1], n),
        np.minimum(np.exp(rng.uniform(np.log(6e4), np.log(1e30), n // 8)), 9e29),
        # within a few ulp of k pi/2 (k >= 1, either sign)
        rng.integers(1, 40000, n) * (np.pi / 2),
    ]
    x = np.concatenate(parts).astype(np.float32)
    near = np.abs(x[-n:]).view(np.int32) + rng.integers(-3, 4, n).astype(np.int32)
    x[-n:] = near.view(np.float32) * rng.choice([-1, 1], n).astype(np.float32)
    assert np.isfinite(x).all() and np.abs(x).max() <= 1e30
    return x


def _ulp_error(got, x, fn):
    with np.errstate(over="ignore", divide="ignore", invalid="ignore"):
        ref = fn(x.astype(np.float64))
        ref32 = ref.astype(np.float32)
        spacing = np.spacing(np.abs(ref32)).astype(np.float64)
        spacing = np.maximum(spacing, np.float64(np.spacing(np.float32(0))))
        err = np.abs(got.astype(np.float64) - ref) / spacing
    both_inf = np.isinf(ref32) & np.isinf(got) & (np.sign(ref32) == np.sign(got))
    return np.where(both_inf, 0.0, err)


def _eval_one(op, x):
    y = np.linspace(-1, 1, len(x)).astype(np.float32)
    ds = beagle.Dataset(x[None, :], y)
    dp = beagle.DevicePrograms(S.from_token_lists([[(S.LOAD0, 0.0), (op, 0.0)]]))
    outs, _ = beagle.eval_programs(dp, ds)
    got = outs[0].cpu().numpy()
    ds.release()
    return got


def _plog64(x):
    a = np.abs(x)
    with np.errstate(divide="ignore"):
        return np.where(a > np.float32(1e-3), np.log(a), 0.0)


@pytest.mark.parametrize("op,fn", [(S.SIN, np.sin), (S.COS, np.cos)])
def test_sin_cos_within_two_ulp(op, fn):
    x = _arguments()
    got = _eval_one(op, x)
    err = _ulp_error(got, x, fn)
    worst = int(np.argmax(err))
    assert err.max() <= 2.0, (float(x[worst]), float(got[worst]), float(err[worst]))
    assert np.median(err) <= 0.5


def test_exp_within_two_ulp():
    rng = np.random.default_rng(7)
    n = 1 << 20
    x = np.concatenate([rng.uniform(-110, 95, n), rng.uniform(-1, 1, n),
                        rng.uniform(-0.4, 0.4, n), rng.uniform(60, 75, n),
                        rng.uniform(-104, -86, n),
                        np.exp(rng.uniform(np.log(1e-30), 0, n)) * rng.choice([-1, 1], n),
                        [0.0, -0.0, 88.72, 88.73, -103.9, -87.4]]).astype(np.float32)
    got = _eval_one(S.EXP, x)
    err = _ulp_error(got, x, np.exp)
    worst = int(np.argmax(err))
    assert err.max() <= 2.0, (float(x[worst]), float(got[worst]), float(err[worst]))
    assert np.isinf(got[x > 88.73]).all() and (got[x < -104] == 0).all()


def test_protected_log_within_two_ulp():
    rng = np.random.default_rng(8)
    n = 1 << 20
    x = np.concatenate([np.exp(rng.uniform(np.log(1e-3), np.log(1e30), n)),
                        rng.uniform(0.5, 2.0, n), rng.uniform(0.99, 1.01, n),
                        rng.uniform(0, 2e-3, n), np.exp(rng.uniform(np.log(1e-30), -6, n))])
    x = np.minimum(x, 9e29) * rng.choice([-1, 1], len(x))
    x = np.concatenate([x, [1e-3, -1e-3, 1.0, -1.0, 2.0, 0.5, 0.0]]).astype(np.float32)
    got = _eval_one(S.PLOG, x)
    err = _ulp_error(got, x, _plog64)
    worst = int(np.argmax(err))
    assert err.max() <= 2.0, (float(x[worst]), float(got[worst]), float(err[worst]))
    assert (got[np.abs(x) <= np.float32(1e-3)] == 0).all()


def test_transcendentals_same_bits_for_every_cases_per_lane():
    x = _arguments(n=1 << 14, seed=3)
    x = np.concatenate([x, np.linspace(-100, 88, 1 << 14, dtype=np.float32)])
    y = np.linspace(-1, 1, len(x)).astype(np.float32)
    ds = beagle.Dataset(x[None, :], y)
    progs = S.from_token_lists([[(S.LOAD0, 0.0), (op, 0.0)]
                                for op in (S.SIN, S.COS, S.EXP, S.PLOG)])
    dp = beagle.DevicePrograms(progs)
    ref = None
    try:
        for cases in (4, 2, 8):
            beagle.set_launch_config(cases_per_lane=cases, tile=512)
            outs, _ = beagle.eval_programs(dp, ds)
            o = outs.cpu().numpy()
            if ref is None:
                ref = o
            else:
                assert np.array_equal(o, ref)
    finally:
        beagle.reset_launch_config()
    ds.release()
