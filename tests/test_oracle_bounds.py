"""Pins of the oracle's running error bound (no GPU): a device model that perturbs every
sin, cos, exp and log result by up to the documented ulp error must land inside the bound;
programs without transcendentals have a zero per-case bound, and their fitness bound (the
aggregation slack alone) covers the same outputs aggregated by tiles in the device's fp64
order."""
from __future__ import annotations

import math

import numpy as np

import oracle
from paper_2607_06731_gb300 import synth as S


def _perturbed(ops, cs, x, rng):
    """FP32-ops evaluation with each transcendental result moved by a random number of ulps
    within oracle.DEV_ULPS_FP32 (a model of a less accurate device library)."""
    st = []
    t = np.float32(1e-3)
    for o, c in zip(ops, cs):
        o = int(o)
        if o >= S.LOAD0:
            st.append(np.float32(x[o - S.LOAD0]))
            continue
        if o == S.CONST:
            st.append(np.float32(c))
            continue
        if o in S.BINARY:
            b, a = st.pop(), st.pop()
            with np.errstate(all="ignore"):
                r = (a + b if o == S.ADD else a - b if o == S.SUB else a * b if o == S.MUL
                     else (a / b if abs(b) > t else np.float32(1)))
            st.append(np.float32(r))
            continue
        a = st.pop()
        if o == S.PSQRT:
            st.append(np.sqrt(np.abs(a)))
            continue
        if o == S.SQUARE:
            with np.errstate(all="ignore"):
                st.append(np.float32(a * a))
            continue
        try:
            v = {S.SIN: math.sin, S.COS: math.cos, S.EXP: math.exp}[o](float(a)) \
                if o != S.PLOG else (math.log(abs(float(a))) if abs(a) > t else 0.0)
        except OverflowError:
            v = math.inf
        with np.errstate(all="ignore"):
            r = np.float32(v)
        if o != S.PLOG or abs(a) > t:
            k = int(rng.integers(-int(oracle.DEV_ULPS_FP32[o]), int(oracle.DEV_ULPS_FP32[o]) + 1))
            for _ in range(abs(k)):
                r = np.nextafter(r, np.float32(math.inf if k > 0 else -math.inf))
        st.append(r)
    return float(st[0])


def test_bound_contains_perturbed_evaluations():
    pr = S.make_c1(P=120, N=40)
    rng = np.random.default_rng(0)
    checked = 0
    for p in range(pr.programs.P):
        ops, cs = pr.programs.program(p)
        f, dl, fl = oracle.eval_bound(ops, cs, pr.X, "fp32")
        if fl & (oracle.F_INVALID | oracle.F_AMBIG):
            continue
        for i in range(pr.N):
            for _ in range(6):
                g = _perturbed(ops, cs, pr.X[:, i], rng)
                assert abs(g - f[i]) <= dl[i] * (1 + 1e-6) + 1e-30, (p, i, g, f[i], dl[i])
                checked += 1
    assert checked > 10000


def test_bound_is_zero_without_transcendentals():
    rng = np.random.default_rng(1)
    X = rng.uniform(-3, 3, size=(2, 64)).astype(np.float32)
    progs = S.gen_programs(rng, 100, 3, 40, 2, unary=(S.SQUARE, S.PSQRT))
    for p in range(progs.P):
        ops, cs = progs.program(p)
        f, dl, fl = oracle.eval_bound(ops, cs, X, "fp32")
        if fl & oracle.F_INVALID:
            continue
        assert np.all(dl == 0.0)
        f2, _ = oracle.eval_program(ops, cs, X, "fp32")
        assert np.array_equal(f, f2)


def test_fitness_bound_covers_perturbed_fitness():
    pr = S.make_c1(P=60, N=50)
    rng = np.random.default_rng(2)
    m, r, fl, bm, br = oracle.score_bound(pr.programs, pr.X, pr.y, "fp32")
    for p in range(pr.programs.P):
        if fl[p] & (oracle.F_INVALID | oracle.F_AMBIG):
            continue
        ops, cs = pr.programs.program(p)
        for _ in range(5):
            g = np.array([_perturbed(ops, cs, pr.X[:, i], rng) for i in range(pr.N)])
            mg, rg, _ = oracle.aggregate(g, pr.y)
            assert abs(mg - m[p]) <= bm[p] * (1 + 1e-6) + 1e-12 * abs(m[p]), p
            if not (fl[p] & oracle.F_DEGENERATE) and np.any(g != g[0]):
                assert abs(rg - r[p]) <= br[p] * (1 + 1e-6) + 1e-12, p


def _tiled_omr2(f, y, tile=512):
    """1 - r^2 aggregated the way a tiled device does it in fp64, in an order unlike the
    oracle's: per tile a two-pass mean m_t and the sums of d = f - m_t, d^2 and d (y - ybar),
    plain fp64; the tiles merged around fbar = sum (n_t m_t + sum d) / N with
    S_ff = sum (sum d^2 + 2 (m_t - fbar) sum d + n_t (m_t - fbar)^2) and
    S_fy = sum (sum d (y - ybar) + (m_t - fbar) sum (y - ybar))."""
    f = np.asarray(f, np.float64)
    yd = np.asarray(y, np.float64)
    yc = yd - yd.sum() / len(yd)
    tiles = []
    for a in range(0, len(f), tile):
        ft, yt = f[a:a + tile], yc[a:a + tile]
        m = ft.sum() / len(ft)
        d = ft - m
        tiles.append((len(ft), m, d.sum(), float(np.dot(d, d)), float(np.dot(d, yt)), yt.sum()))
    fbar = sum(n * m + sd for n, m, sd, _, _, _ in tiles) / len(f)
    sff = sum(sdd + 2.0 * (m - fbar) * sd + n * (m - fbar) ** 2 for n, m, sd, sdd, _, _ in tiles)
    sfy = sum(sdy + (m - fbar) * sy for _, m, _, _, sdy, sy in tiles)
    syy = float(np.dot(yc, yc))
    return 1.0 - sfy * sfy / (sff * syy)


def test_aggregation_slack_covers_a_tiled_fp64_aggregation():
    """For programs without transcendentals every per-case bound is 0 (both sides round the
    same correctly rounded operations), so the 1 - r^2 bound is the aggregation slack alone:
    it must cover the same outputs aggregated by tiles in another fp64 order -- including
    outputs that differ only in their last bits, where the rounding of the mean dominates."""
    rng = np.random.default_rng(31)
    N = 3000
    X = rng.uniform(-2, 2, (2, N)).astype(np.float32)
    y = (X[0] * X[1] + 0.3 * X[0]).astype(np.float32)
    progs = S.gen_programs(rng, 300, 3, 30, 2, unary=(S.SQUARE,))
    C, L0 = S.CONST, S.LOAD0
    # outputs 1 + x0 1e-14 and 1e6 + x1: variation only in the last bits of the fp64 outputs
    near = S.from_token_lists([[(L0, 0.0), (C, 1e-14), (S.MUL, 0.0), (C, 1.0), (S.ADD, 0.0)],
                               [(L0 + 1, 0.0), (C, 1e6), (S.ADD, 0.0)]])
    for pop in (progs, near):
        m, r, fl, bm, br = oracle.score_bound(pop, X, y, "fp64")
        checked = 0
        for p in range(pop.P):
            if fl[p] & (oracle.F_INVALID | oracle.F_DEGENERATE | oracle.F_MALFORMED):
                continue
            ops, cs = pop.program(p)
            f, _ = oracle.eval_program(ops, cs, X, "fp64")
            if np.all(f == f[0]):
                assert br[p] == 0.0
                continue
            assert br[p] > 0.0                      # the slack, per-case bounds being 0
            for tile in (512, 256):
                got = _tiled_omr2(f, y, tile)
                assert abs(got - r[p]) <= br[p], (p, tile, got, r[p], br[p])
            checked += 1
        assert checked >= (2 if pop is near else 100)
