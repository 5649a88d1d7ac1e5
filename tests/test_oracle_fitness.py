"""Pins of the oracle's versions of the paper's fitness functions (oracle_fit_*): the
correlation score of Eq. 2, the point-to-point family of Eq. 5, the validation test of the
interactive V command and the length tax, against values worked by hand, numpy's correlation
and brute-force counting written here independently."""
from __future__ import annotations

import math

import numpy as np
import pytest

import oracle
from paper_2607_06731_gb300 import synth as S

M = 10_000
MODES = ("fp32", "fp64")


def prog(*toks):
    return S.from_token_lists([list(toks)])


X0 = (S.LOAD0, 0.0)
X1 = (S.LOAD0 + 1, 0.0)
MUL = (S.MUL, 0.0)


def fit(progs, X, y, kind, mode, M=M, tax=0.0):
    out, cnt, flags = oracle.fit_score(progs, np.asarray(X, np.float32), np.asarray(y, np.float32),
                                       kind, M, mode, tax)
    return out, cnt, flags


@pytest.mark.parametrize("mode", MODES)
def test_correlation_hand_case_with_invalid_pairs(mode):
    """x0 * x0 on six cases: two valid/valid pairs with f == y plus one more, one pair where
    both are invalid (square above 1e30, target NaN), two with exactly one invalid."""
    X = [[1, 2, 1e20, 1e16, 3, 4]]
    y = [1, 4, np.nan, 7, np.nan, 16]
    out, cnt, flags = fit(prog(X0, X0, MUL), X, y, oracle.FIT_CORRELATION, mode)
    assert list(cnt[0]) == [2, 1]                 # c1: cases 3 and 4; c2: case 2
    # valid pairs (1,1), (4,4), (16,16): r = 1 exactly; score = M (6 - 3) - M (2 - 1) = 2M
    assert out[0, 0] == 2 * M and out[0, 2] == 1.0
    assert out[0, 1] == pytest.approx(2 * M / (M * 6), abs=0)
    assert flags[0] & oracle.F_DEGENERATE == 0


@pytest.mark.parametrize("mode", MODES)
def test_correlation_r_one_half(mode):
    """f = (1, 2, 3), y = (1, 3, 2): deviations (-1, 0, 1) and (-1, 1, 0) give S_fy = 1,
    S_ff = S_yy = 2, r = 1/2, r^4 = 1/16: score = M * 3 / 16."""
    out, cnt, _ = fit(prog(X0), [[1, 2, 3]], [1, 3, 2], oracle.FIT_CORRELATION, mode)
    assert out[0, 0] == M * 3 / 16 and out[0, 2] == 0.25 and list(cnt[0]) == [0, 0]


def test_correlation_matches_numpy_without_invalids():
    rng = np.random.default_rng(1)
    X = rng.uniform(-2, 2, (3, 700)).astype(np.float32)
    y = (X[0] * X[1] + rng.normal(0, 0.3, 700)).astype(np.float32)
    progs = S.gen_programs(rng, 60, 3, 30, 3)
    out, cnt, flags = fit(progs, X, y, oracle.FIT_CORRELATION, "fp64")
    for p in range(progs.P):
        ops, cs = progs.program(p)
        f, fl = oracle.eval_program(ops, cs, X, "fp64")
        if fl & oracle.F_INVALID:
            assert cnt[p, 0] > 0
            continue
        assert list(cnt[p]) == [0, 0]
        if np.all(f == f[0]):
            assert flags[p] & oracle.F_DEGENERATE and out[p, 0] == 0.0
            continue
        if np.std(f) <= 1e-9 * abs(np.mean(f)):
            continue    # outputs differing in their last bits only: r is rounding noise
        r = np.corrcoef(f, y.astype(np.float64))[0, 1]
        assert out[p, 2] == pytest.approx(r * r, rel=1e-11, abs=1e-14)
        assert out[p, 0] == pytest.approx(M * r ** 4 * 700, rel=1e-10, abs=1e-9)


def test_correlation_counts_against_brute_force():
    """Random NaN / inf / oversized targets and overflowing programs: c1, c2 and r over the
    valid pairs, counted and correlated here case by case."""
    rng = np.random.default_rng(2)
    N = 400
    X = rng.uniform(-30, 30, (2, N)).astype(np.float32)
    y = (X[0] * 0.5 + rng.normal(0, 1, N)).astype(np.float32)
    bad_t = rng.random(N) < 0.15
    y[bad_t] = rng.choice([np.nan, np.inf, -np.inf, 3e30], bad_t.sum()).astype(np.float32)
    # exp(x0) overflows 1e30 for x0 > 69.08; x0 * 3 keeps some cases valid
    progs = S.from_token_lists([[X0, (S.CONST, 3.0), MUL, (S.EXP, 0.0)],
                                [X0, (S.EXP, 0.0), X1, (S.ADD, 0.0)],
                                [X0, X0, MUL, X0, MUL, X0, MUL, X0, MUL]])
    out, cnt, _ = fit(progs, X, y, oracle.FIT_CORRELATION, "fp64")
    yd = y.astype(np.float64)
    tv = np.abs(yd) <= 1e30
    for p in range(progs.P):
        ops, cs = progs.program(p)
        f, bad, _ = oracle.eval_cases(ops, cs, X, "fp64")
        # independent per-case validity: recompute the program's values with numpy
        x0, x1 = X[0].astype(np.float64), X[1].astype(np.float64)
        if p == 0:
            fv = np.abs(np.exp(x0 * 3)) <= 1e30
            ref = np.exp(x0 * 3)
        elif p == 1:
            fv = np.abs(np.exp(x0)) <= 1e30
            ref = np.exp(x0) + x1
        else:
            vals = [x0 * x0, x0 ** 3, x0 ** 4, x0 ** 5]
            fv = np.all([np.abs(v) <= 1e30 for v in vals], axis=0)
            ref = x0 ** 5
        assert np.array_equal(bad == 0, fv)
        c1 = int(np.sum(fv != tv))
        c2 = int(np.sum(~fv & ~tv))
        assert list(cnt[p]) == [c1, c2]
        V = fv & tv
        r = np.corrcoef(ref[V], yd[V])[0, 1]
        n = int(V.sum())
        assert n == N - c1 - c2
        assert out[p, 2] == pytest.approx(r * r, rel=1e-9)
        assert out[p, 0] == pytest.approx(M * r ** 4 * n - M * (c1 - c2), rel=1e-9, abs=1e-6)


@pytest.mark.parametrize("mode", MODES)
def test_correlation_degenerate_output(mode):
    """A constant program: r is undefined, read as 0; the score keeps its c1/c2 term."""
    y = [1, 2, np.nan, 4]
    out, cnt, flags = fit(prog((S.CONST, 1.5)), [[0, 0, 0, 0]], y, oracle.FIT_CORRELATION, mode)
    assert flags[0] & oracle.F_DEGENERATE and out[0, 2] == 0.0
    assert list(cnt[0]) == [1, 0] and out[0, 0] == -M


def std_case(f, y, kind, mode, M=M):
    """Reward of one valid pair: program x0 * x1 with x1 = 1 gives f exactly."""
    out, _, _ = fit(prog(X0, X1, MUL), [[f], [1.0]], [y], kind, mode, M=M)
    return out[0, 0]


@pytest.mark.parametrize("mode", MODES)
def test_std_family_hand_values(mode):
    K = (oracle.FIT_STD, oracle.FIT_STD_SQUARE, oracle.FIT_STD_CUBE, oracle.FIT_STD_HYPER)
    # same signs, q = 1/2: M q^k rounded; M/2^8 = 39.0625 -> 39
    assert [std_case(2, 4, k, mode) for k in K] == [5000, 2500, 1250, 39]
    # opposite signs: M q^k - M/11 (909.0909...) rounded
    assert [std_case(-2, 4, k, mode) for k in K] == [4091, 1591, 341, -870]
    assert std_case(-0.01, 1, oracle.FIT_STD, mode) == -809      # 100 - 909.09
    assert std_case(0, 0, oracle.FIT_STD, mode) == M             # both zero: M
    assert std_case(3, 3, oracle.FIT_STD_HYPER, mode) == M       # exact fit
    # ties round to even: M = 10, q = 1/4 -> 2.5 -> 2; q = 3/4 -> 7.5 -> 8
    assert std_case(1, 4, oracle.FIT_STD, mode, M=10) == 2
    assert std_case(3, 4, oracle.FIT_STD, mode, M=10) == 8


@pytest.mark.parametrize("mode", MODES)
def test_std_invalid_pairs_and_sum(mode):
    """Per-case rewards add up; an invalid output (1e10 * 1e30 > 1e30) against a valid target
    costs M, against an invalid target earns M; a valid output against an invalid target
    costs M."""
    X = [[2, 1e10, 1e10, 2], [1, 1e30, 1e30, 1]]
    y = [4, 4, np.nan, np.nan]
    out, cnt, _ = fit(prog(X0, X1, MUL), X, y, oracle.FIT_STD, mode)
    assert out[0, 0] == 5000 - M + M - M and list(cnt[0]) == [2, 1]
    assert out[0, 1] == (5000 - M) / (M * 4)


@pytest.mark.parametrize("mode", MODES)
def test_std_brute_force(mode):
    """Random valid pairs: the sum of Eq. 5 rewards computed here one pair at a time."""
    rng = np.random.default_rng(3)
    N = 300
    f = rng.uniform(-5, 5, N).astype(np.float32)
    f[::17] = 0
    y = rng.uniform(-5, 5, N).astype(np.float32)
    y[::23] = 0
    for kind, k in ((oracle.FIT_STD, 1), (oracle.FIT_STD_SQUARE, 2), (oracle.FIT_STD_CUBE, 3),
                    (oracle.FIT_STD_HYPER, 8)):
        out, _, _ = fit(prog(X0, X1, MUL), [f, np.ones(N, np.float32)], y, kind, mode)
        tot = 0
        for a, b in zip(f, y):
            if mode == "fp32":
                a32, b32 = np.float32(abs(a)), np.float32(abs(b))
                mx, mn = max(a32, b32), min(a32, b32)
                if mx == 0:
                    tot += M
                    continue
                q = np.float32(mn / mx)
                qk = {1: q, 2: np.float32(q * q), 3: np.float32(np.float32(q * q) * q),
                      8: np.float32(np.float32(np.float32(q * q) ** 2) ** 2)}[k]
                v = np.float32(np.float32(M) * qk)
                if (a < 0 < b) or (b < 0 < a):
                    v = np.float32(v - np.float32(np.float32(M) / np.float32(11)))
                tot += int(np.rint(v))
            else:
                mx, mn = max(abs(float(a)), abs(float(b))), min(abs(float(a)), abs(float(b)))
                if mx == 0:
                    tot += M
                    continue
                q = mn / mx
                qk = {1: q, 2: q * q, 3: (q * q) * q, 8: ((q * q) ** 2) ** 2}[k]
                v = M * qk
                if (a < 0 < b) or (b < 0 < a):
                    v = v - M / 11
                tot += int(np.rint(v))
        assert out[0, 0] == tot


@pytest.mark.parametrize("mode", MODES)
def test_validation_test(mode):
    """The V command's test: within 0.1 % of the target on every case."""
    X = [[100, 100.05, 100.2, 0, 5]]
    y = [100, 100, 100, 0, np.nan]
    out, cnt, flags = fit(prog(X0), X, y, oracle.FIT_VALIDATE, mode)
    assert out[0, 0] == 3 and out[0, 1] == 3 / 5 and not flags[0] & oracle.F_PERFECT
    out, _, flags = fit(prog(X0), [[1, -2, 3.0015]], [1, -2, 3], oracle.FIT_VALIDATE, mode)
    assert out[0, 0] == 3 and flags[0] & oracle.F_PERFECT


def test_length_tax_default_rate():
    """ScriptLengthTaxRateInternal's default, M N / 85: a perfect program of length 85 is
    taxed to zero. x0 then 42 (DUP, DEL) pairs is 85 tokens and returns x0."""
    toks = [X0] + [(S.DUP, 0.0), (S.DEL, 0.0)] * 42
    X = [[1, 2, -3, 4]]
    out, _, _ = fit(prog(*toks), X, X[0], oracle.FIT_STD, "fp64", tax=-1.0)
    assert out[0, 0] == M * 4
    assert abs(out[0, 3]) <= 1e-9 * M * 4
    out, _, _ = fit(prog(*toks), X, X[0], oracle.FIT_STD, "fp64", tax=10.0)
    assert out[0, 3] == M * 4 - 850


def test_malformed_program_scores_minus_infinity():
    out, _, flags = fit(prog(X0, MUL), [[1, 2]], [1, 2], oracle.FIT_CORRELATION, "fp64")
    assert flags[0] & oracle.F_MALFORMED and out[0, 0] == -math.inf
