"""The early exit on invalid programs (GPU): a program with an invalid value on one case is
invalid whatever its other cases give, so a case tile stops at the first pass that meets one
and the later tiles of a program found invalid are not run. The scores must be the bits that
running every case gives, and the per-program case counts must show what ran: every case of a
valid program, fewer for invalid ones, none for malformed ones."""
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
    beagle.set_invalid_early_exit(True)
    beagle.count_cases(None)
    beagle.reset_launch_config()


def _concat(a, b):
    return S.Programs(np.concatenate([a.ops, b.ops]),
                      np.concatenate([a.offsets, b.offsets + len(a.ops)]),
                      np.concatenate([a.lengths, b.lengths]), np.concatenate([a.consts, b.consts]))


def _population(rng, d):
    """Random programs over the whole operator set on wide inputs (many overflow somewhere),
    programs invalid only on the last cases (exp(c x0) with x0 sorted: only the largest x0
    overflow), valid ones, and malformed ones."""
    P0 = S.gen_programs(rng, 500, 4, 60, d, unary=S.ALL_UNARY, binary=S.ALL_BINARY)
    L0, C = S.LOAD0, S.CONST
    late = [[(L0, 0.0), (C, c), (S.MUL, 0.0), (S.EXP, 0.0)] for c in (13.0, 14.0, 15.0)]
    valid = [[(L0 + 1, 0.0), (S.SIN, 0.0)], [(L0, 0.0), (L0 + 2, 0.0), (S.MUL, 0.0)]]
    bad = [[(S.ADD, 0.0)], [(C, 1.0), (C, 2.0)]]
    return _concat(P0, S.from_token_lists(late + valid + bad))


def _score(dp, ds, P, precision, early):
    beagle.set_invalid_early_exit(early)
    counts = torch.zeros(P, dtype=torch.int64, device="cuda")
    beagle.count_cases(counts)
    try:
        out = beagle.score_programs(dp, ds, precision=precision)
        torch.cuda.synchronize()
    finally:
        beagle.count_cases(None)
        beagle.set_invalid_early_exit(True)
    return beagle.unpack_fitness(out), counts.cpu().numpy()


@pytest.mark.parametrize("cases,keep_order", [(4, 2), (4, 1), (8, 2), (2, 1)])
def test_early_exit_same_bits_and_case_counts(cases, keep_order):
    rng = np.random.default_rng(500 + cases + 10 * keep_order)
    d, N = 3, 5000                       # 10 tiles of 512 cases, a ragged last one
    X = rng.uniform(-6, 6, (d, N)).astype(np.float32)
    X[0] = np.sort(X[0])                 # the largest x0 in the last tile
    y = (X[0] * X[1] + np.sin(X[2])).astype(np.float32)
    progs = _population(rng, d)
    P = progs.P
    ds = beagle.Dataset(X, y)
    dp = beagle.DevicePrograms(progs)
    beagle.set_launch_config(cases_per_lane=cases, keep_order=keep_order)
    try:
        for precision in ("fp32c", "fp64"):
            on, n_on = _score(dp, ds, P, precision, True)
            off, n_off = _score(dp, ds, P, precision, False)
            for a, b in zip(on, off):
                assert np.array_equal(a, b, equal_nan=True)
            flags = on[2]
            malformed = (flags & beagle.FLAG_MALFORMED) != 0
            invalid = (flags & beagle.FLAG_INVALID) != 0
            assert malformed.sum() == 2 and invalid.sum() > 50 and (~invalid & ~malformed).sum() > 50
            assert np.all(n_off[~malformed] == N) and np.all(n_off[malformed] == 0)
            assert np.all(n_on[~invalid & ~malformed] == N)
            assert np.all(n_on[malformed] == 0)
            assert np.all(n_on[invalid] <= N) and np.any(n_on[invalid] < N // 2)
            # the late-overflow programs are invalid and stop only in the last tiles
            late = np.arange(500, 503)
            assert np.all(invalid[late]) and np.all(n_on[late] > N // 2)
            assert np.all(n_on[late] < N)
            if precision == "fp32c" and cases == 4:
                parity.check_fp32(on, parity.references(progs, X, y), name="early-exit")
    finally:
        beagle.reset_launch_config()
        ds.release()


def test_case_counter_needs_a_positive_population():
    with pytest.raises(beagle.BeagleError):
        beagle.check(beagle.lib().beagle_count_cases(1, 0))


@pytest.mark.parametrize("precision", ["fp32c", "fp64"])
def test_serving_early_exit_same_bits(precision):
    """The serving loop stops invalid programs early too (the setting taken per request): the
    served records are the bits served with every case run, and beagle_score's."""
    rng = np.random.default_rng(620)
    d, N = 3, 3000
    X = rng.uniform(-6, 6, (d, N)).astype(np.float32)
    X[0] = np.sort(X[0])
    y = (X[0] * X[1] + np.sin(X[2])).astype(np.float32)
    progs = _population(rng, d)
    ds = beagle.Dataset(X, y)
    try:
        ref, _ = _score(beagle.DevicePrograms(progs), ds, progs.P, precision, True)
        served = []
        for early in (True, False):
            beagle.set_invalid_early_exit(early)
            srv = beagle.Server(precision=precision)
            try:
                served.append(beagle.unpack_fitness(srv.wait(srv.submit(progs, ds),
                                                             timeout_us=60_000_000)))
            finally:
                srv.destroy()
                beagle.set_invalid_early_exit(True)
        for got in served:
            for a, b in zip(got, ref):
                assert np.array_equal(a, b, equal_nan=True)
        assert np.any(ref[2] & beagle.FLAG_INVALID)
    finally:
        ds.release()
