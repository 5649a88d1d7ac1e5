"""The rest of Table 3 on the GPU (POW, SIGN, CUBE, CBRT, TAN, ARCSIN, ARCCOS, ARCTAN, TANH and
the COPY/PASTE variables) against the oracle with its error bound, in both precisions and
every cases-per-lane variant; and the accuracy of the new transcendentals against the ulp
limits the oracle's bound assumes (oracle.DEV_ULPS_FP32 / FP64)."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_2607_06731_gb300 import beagle, synth as S
from tests import parity

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    beagle.reset_launch_config()
    yield
    beagle.reset_launch_config()


def _gpu(progs, ds, precision):
    dp = beagle.DevicePrograms(progs)
    out = beagle.score_programs(dp, ds, precision=precision)
    torch.cuda.synchronize()
    return beagle.unpack_fitness(out)


def _programs(seed, P=600, d=3):
    rng = np.random.default_rng(seed)
    base = S.gen_programs(rng, P, 2, 40, d, unary=S.ALL_UNARY, binary=S.ALL_BINARY,
                          depth_cap=12)
    return S.with_registers(base, rng, frac=0.5, n_regs=2)


@pytest.mark.parametrize("N", [700, 1500])
@pytest.mark.parametrize("cases", [4, 2, 8])
def test_full_op_set_matches_the_oracle(N, cases):
    rng = np.random.default_rng(N + 7 * cases)
    d = 3
    X = rng.uniform(-1.5, 1.5, (d, N)).astype(np.float32)
    y = (np.tanh(X[0]) + X[1] * X[2]).astype(np.float32)
    progs = _programs(N + cases, d=d)
    assert beagle.validate_programs(progs.ops, progs.offsets, progs.lengths, d) == -1
    refs = parity.references(progs, X, y)
    ds = beagle.Dataset(X, y)
    beagle.set_launch_config(cases_per_lane=cases)
    try:
        g32 = _gpu(progs, ds, "fp32c")
        parity.check_fp32(g32, refs, name=f"ops-{cases}-{N}")
        if cases == 4:
            g64 = _gpu(progs, ds, "fp64")
            parity.check_fp64(g64, refs, name=f"ops-{N}")
    finally:
        beagle.reset_launch_config()
        ds.release()


def _eval(progs, X, precision):
    y = np.linspace(-1, 1, X.shape[1]).astype(np.float32)
    ds = beagle.Dataset(X, y)
    dp = beagle.DevicePrograms(progs)
    outs, _ = beagle.eval_programs(dp, ds, precision=precision)
    torch.cuda.synchronize()
    ds.release()
    return outs.cpu().numpy()


def _ulps32(got, exact):
    """|got - exact| in units of the fp32 spacing at the exact value."""
    e32 = exact.astype(np.float32)
    sp = np.spacing(np.abs(e32)).astype(np.float64)
    return np.abs(got.astype(np.float64) - exact) / sp


@pytest.mark.parametrize("op,lo,hi,fn", [
    (S.CBRT, -1e6, 1e6, np.cbrt), (S.TAN, -10.0, 10.0, np.tan),
    (S.TAN, -3e4, 3e4, np.tan), (S.ASIN, -1.0, 1.0, np.arcsin),
    (S.ACOS, -1.0, 1.0, np.arccos), (S.ATAN, -1e5, 1e5, np.arctan),
    (S.TANH, -12.0, 12.0, np.tanh)])
def test_new_transcendentals_within_their_ulp_limits(op, lo, hi, fn):
    rng = np.random.default_rng(op)
    n = 1 << 18
    x = rng.uniform(lo, hi, n).astype(np.float32)
    x[: n // 8] = (x[: n // 8] * 1e-3).astype(np.float32)   # small arguments too
    progs = S.from_token_lists([[(S.LOAD0, 0.0), (op, 0.0)]])
    exact = fn(x.astype(np.float64))
    got32 = _eval(progs, x[None, :], "fp32c")[0]
    u = _ulps32(got32, exact)
    fin = np.isfinite(exact) & (np.abs(exact) > 1e-30)
    assert np.max(u[fin]) <= oracle.DEV_ULPS_FP32[op], (S.NAMES[op], float(np.max(u[fin])))
    got64 = _eval(progs, x[None, :], "fp64")[0]
    sp64 = np.spacing(np.abs(exact))
    u64 = np.abs(got64 - exact) / sp64
    # numpy's own value is within about an ulp of the exact one
    assert np.max(u64[fin]) <= oracle.DEV_ULPS_FP64[op] + 1, (S.NAMES[op], float(np.max(u64[fin])))


def test_pow_within_its_ulp_limit():
    rng = np.random.default_rng(3)
    n = 1 << 18
    a = np.exp(rng.uniform(np.log(1e-3), np.log(1e3), n)).astype(np.float32)
    b = rng.uniform(-8, 8, n).astype(np.float32)
    a[: n // 4] = -a[: n // 4]                       # negative bases with integer exponents
    b[: n // 4] = np.round(b[: n // 4])
    progs = S.from_token_lists([[(S.LOAD0, 0.0), (S.LOAD0 + 1, 0.0), (S.POW, 0.0)]])
    X = np.stack([a, b])
    exact = np.power(a.astype(np.float64), b.astype(np.float64))
    fin = np.isfinite(exact) & (np.abs(exact) > 1e-30) & (np.abs(exact) < 1e30)
    got32 = _eval(progs, X, "fp32c")[0]
    assert np.max(_ulps32(got32, exact)[fin]) <= oracle.DEV_ULPS_FP32[S.POW]
    got64 = _eval(progs, X, "fp64")[0]
    assert np.max((np.abs(got64 - exact) / np.spacing(np.abs(exact)))[fin]) <= \
        oracle.DEV_ULPS_FP64[S.POW] + 1


def test_ieee_new_ops_are_exact():
    """SIGN and CUBE are correctly rounded fp32 operations: the same bits as numpy float32;
    COPY/PASTE move values without arithmetic."""
    rng = np.random.default_rng(4)
    x = rng.uniform(-40, 40, 4096).astype(np.float32)
    z = rng.uniform(-3, 3, 4096).astype(np.float32)
    progs = S.from_token_lists([
        [(S.LOAD0, 0.0), (S.SIGN, 0.0)],
        [(S.LOAD0, 0.0), (S.CUBE, 0.0)],
        [(S.LOAD0, 0.0), (S.COPY0 + 2, 0.0), (S.LOAD0 + 1, 0.0), (S.ADD, 0.0),
         (S.PASTE0 + 2, 0.0), (S.MUL, 0.0)]])
    for prec, dt in (("fp32c", np.float32), ("fp64", np.float64)):
        out = _eval(progs, np.stack([x, z]), prec)
        xx, zz = x.astype(dt), z.astype(dt)
        assert np.array_equal(out[0], -xx)
        assert np.array_equal(out[1], (xx * xx) * xx)
        assert np.array_equal(out[2], (xx + zz) * xx)


def test_register_and_stack_share_the_gpu_limit():
    """A live variable k takes stack row D - 2 - k on the GPU: a program whose depth plus
    (k + 1) passes the fast pass's 16 runs in the deep pass (32), and one that passes 32 is
    flagged MALFORMED, while the oracle (variables apart from its 32-value stack) runs it."""
    X = np.linspace(0.5, 1.5, 300, dtype=np.float32)[None, :]
    y = X[0] * 2

    def prog(k, depth):
        return [(S.LOAD0, 0.0), (S.COPY0 + k, 0.0)] + [(S.CONST, 1.0)] * (depth - 1) + \
               [(S.ADD, 0.0)] * (depth - 1) + [(S.PASTE0 + k, 0.0), (S.ADD, 0.0)]
    progs = S.from_token_lists([prog(0, 15), prog(1, 15), prog(1, 30), prog(2, 30)])
    ds = beagle.Dataset(X, y)
    g = _gpu(progs, ds, "fp32c")
    ds.release()
    o = oracle.score_programs(progs, X, y, "fp32")
    for p in range(3):            # 16 (fast pass), 17 and 32 (deep pass) values in use
        assert g[2][p] == o[2][p] == 0 and g[0][p] == pytest.approx(o[0][p], rel=1e-6), p
    assert g[2][3] & beagle.FLAG_MALFORMED and not o[2][3] & oracle.F_MALFORMED   # 33
