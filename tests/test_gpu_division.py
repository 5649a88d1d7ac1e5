"""The FP32 protected division against IEEE float32 division, through the interpreter.

The FP32 paths divide by Markstein's method (a refined reciprocal approximation and one
remainder correction). Its remainder num - den q is exact while it is a normal number, so the
quotient is the correctly rounded one for |num| >= 2^-100 with a normal quotient: every divisor
mantissa is checked exhaustively, then random pairs over a wide exponent range, on each
cases-per-lane variant. Below that (numerators under 2^-100, or subnormal quotients) the
remainder is rounded and the quotient may be one unit in the last place off: that range is
pinned to 1 ulp. Zero quotients may differ from IEEE in the sign of zero only, which numeric
comparison ignores.
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


def _quotients(num: np.ndarray, den: np.ndarray, cases: int) -> np.ndarray:
    """pdiv(num, den) per case: the program x0 x1 PDIV (leaf push, fused divide by input)."""
    X = np.stack([num, den]).astype(np.float32)
    ds = beagle.Dataset(X, np.linspace(0, 1, X.shape[1], dtype=np.float32))
    dp = beagle.DevicePrograms(S.from_token_lists([[(S.LOAD0, 0.0), (S.LOAD0 + 1, 0.0),
                                                    (S.PDIV, 0.0)]]))
    beagle.set_launch_config(cases_per_lane=cases)
    try:
        outs, _ = beagle.eval_programs(dp, ds)
        torch.cuda.synchronize()
        return outs.cpu().numpy()[0]
    finally:
        beagle.reset_launch_config()
        ds.release()


def _ieee(num: np.ndarray, den: np.ndarray) -> np.ndarray:
    with np.errstate(all="ignore"):
        q = num.astype(np.float32) / den.astype(np.float32)
    return np.where(np.abs(den) > np.float32(1e-3), q, np.float32(1.0))


def _check(num, den, cases):
    got = _quotients(num, den, cases)
    want = _ieee(num, den)
    bad = np.nonzero(got != want)[0]
    assert len(bad) == 0, [(float(num[i]), float(den[i]), float(got[i]), float(want[i]))
                           for i in bad[:5]]


@pytest.mark.parametrize("cases", [4, 8, 2])
def test_every_divisor_mantissa(cases):
    """All 2^23 divisor mantissas in [1, 2), with numerators 1 and 1.9999999 and with scaled
    and negated divisors."""
    den = (np.arange(1 << 23, dtype=np.uint32) | np.uint32(0x3F800000)).view(np.float32)
    _check(np.ones_like(den), den, cases)
    _check(np.full_like(den, np.nextafter(np.float32(2), np.float32(0))), -den * 1024, cases)


@pytest.mark.parametrize("cases", [4, 8, 2])
def test_random_pairs(cases):
    """Numerators and divisors with random mantissas and exponents over 2^-60..2^60."""
    rng = np.random.default_rng(7 + cases)
    n = 1 << 22

    def draw():
        m = rng.uniform(1, 2, n) * rng.choice([-1.0, 1.0], n)
        return (m * np.exp2(rng.integers(-60, 61, n))).astype(np.float32)

    _check(draw(), draw(), cases)


def _ulps(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Distance in units in the last place between same-sign finite floats (0 if equal)."""
    ia = a.view(np.int32).astype(np.int64)
    ib = b.view(np.int32).astype(np.int64)
    return np.where(a == b, 0, np.abs(ia - ib))


@pytest.mark.parametrize("cases", [4, 8])
def test_tiny_numerators_within_one_ulp(cases):
    """Numerators 2^-126..2^-100 over divisors 2^-9..2^20: normal quotients whose remainder can
    be subnormal; and quotients down in the subnormal range. At most 1 ulp from IEEE."""
    rng = np.random.default_rng(17 + cases)
    n = 1 << 21
    num = (rng.uniform(1, 2, n) * np.exp2(rng.integers(-126, -99, n))).astype(np.float32)
    den = (rng.uniform(1, 2, n) * rng.choice([-1.0, 1.0], n) *
           np.exp2(rng.integers(-9, 21, n))).astype(np.float32)
    got = _quotients(num, den, cases)
    want = _ieee(num, den)
    assert np.all(np.sign(got) == np.sign(want))
    d = _ulps(np.abs(got), np.abs(want))
    assert d.max() <= 1, int(d.max())
    print(f"cases {cases}: {np.mean(d > 0):.2e} of tiny-numerator quotients 1 ulp off")
