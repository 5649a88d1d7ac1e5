"""The FP32 protected division against IEEE float32 division, through the interpreter.

The FP32 paths divide by Markstein's method (a refined reciprocal approximation and one
remainder correction), which must give the correctly rounded quotient wherever it is a normal
number: every divisor mantissa is checked exhaustively, then random pairs over a wide exponent
range, on each cases-per-lane variant. Zero quotients may differ from IEEE in the sign of zero
only, which numeric comparison ignores.
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
