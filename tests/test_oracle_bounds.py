"""Pins of the oracle's running error bound (no GPU): a device model that perturbs every
sin, cos, exp and log result by up to the documented ulp error must land inside the bound,
and programs without transcendentals have a zero bound."""
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
