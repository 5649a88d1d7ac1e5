"""Pins of the oracle to things other than itself (no GPU needed).

Each test names what fixes the expected value: a value worked out by hand from Table 3,
a closed form, a library routine for a special case, an invariant, or a brute-force
enumeration checked by an evaluator built on a different algorithm.
"""
from __future__ import annotations

import itertools
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_2607_06731_gb300 import synth as S
from tests.gcl_text import paper_genomes

X3 = np.array([[1.0, 2.0, 3.0]], np.float32)


def run(tokens, X=X3, mode="fp64"):
    ops = np.array([t[0] for t in tokens], np.uint8)
    cs = np.array([t[1] for t in tokens], np.float32)
    return oracle.eval_program(ops, cs, X, mode)


def C(v):
    return (S.CONST, v)


def LD(k):
    return (S.LOAD0 + k, 0.0)


def OP(o):
    return (o, 0.0)


# ------------------------------------------------------------------ Table 3, by hand
@pytest.mark.parametrize("mode", ["fp64", "fp32"])
def test_opcode_values_by_hand(mode):
    one = np.array([[0.0]], np.float32)
    cases = [
        ([C(7), C(2), OP(S.ADD)], 9.0),
        ([C(7), C(2), OP(S.SUB)], 5.0),            # second minus top (Table 3 SUB)
        ([C(7), C(2), OP(S.MUL)], 14.0),
        ([C(7), C(2), OP(S.PDIV)], 3.5),           # second divided by top (Table 3 DIV)
        ([C(1), C(0.0005), OP(S.PDIV)], 1.0),      # protected: |b| <= 1e-3 gives 1
        ([C(1), C(-0.0005), OP(S.PDIV)], 1.0),
        ([C(3), C(-0.5), OP(S.PDIV)], -6.0),
        ([C(-3), OP(S.SQUARE)], 9.0),
        ([C(-4), OP(S.PSQRT)], 2.0),               # protected: sqrt |a|
        ([C(0.0005), OP(S.PLOG)], 0.0),            # protected: |a| <= 1e-3 gives 0
        ([C(-1), OP(S.PLOG)], 0.0),                # ln |-1| = 0
        ([C(0), OP(S.EXP)], 1.0),
        ([C(0), OP(S.COS)], 1.0),
        ([C(0), OP(S.SIN)], 0.0),
        ([C(7), C(2), OP(S.SWAP), OP(S.SUB)], -5.0),   # SWAP exchanges the top two
        ([C(7), C(2), OP(S.DEL)], 7.0),                # DEL pops the top
        ([C(3), OP(S.DUP), OP(S.MUL)], 9.0),           # DUP pushes a copy of the top
        ([C(1), C(2), C(3), OP(S.SUB), OP(S.SUB)], 2.0),  # 1 - (2 - 3)
    ]
    for toks, want in cases:
        f, fl = run(toks, one, mode)
        assert fl & ~oracle.F_NEAR == 0, toks
        assert f[0] == want, (toks, f[0], want)


def test_transcendentals_by_hand():
    f, _ = run([C(2), OP(S.PLOG)], np.zeros((1, 1), np.float32))
    assert f[0] == math.log(2.0)
    f, _ = run([C(-2), OP(S.PLOG)], np.zeros((1, 1), np.float32))
    assert f[0] == math.log(2.0)                  # ln |a|
    f, _ = run([C(1), OP(S.EXP)], np.zeros((1, 1), np.float32))
    assert f[0] == math.e
    f, _ = run([C(0.5), OP(S.SIN)], np.zeros((1, 1), np.float32), "fp32")
    assert f[0] == float(np.float32(math.sin(0.5)))


def test_loads_are_zero_based_and_per_case():
    X = np.array([[1, 2, 3], [10, 20, 30]], np.float32)
    f, fl = run([LD(1), LD(0), OP(S.SUB)], X)      # x1 - x0
    assert fl == 0 and list(f) == [9.0, 18.0, 27.0]


# ------------------------------------------------------------------ validity rule
def test_validity_threshold_fp64():
    z = np.zeros((1, 1), np.float32)
    _, fl = run([C(2.0 ** 49), OP(S.SQUARE)], z)   # 2^98 ~ 3.2e29 <= 1e30
    assert fl & oracle.F_INVALID == 0
    _, fl = run([C(2.0 ** 50), OP(S.SQUARE)], z)   # 2^100 ~ 1.27e30 > 1e30
    assert fl & oracle.F_INVALID
    _, fl = run([C(100.0), OP(S.EXP)], z)          # e^100 ~ 2.7e43
    assert fl & oracle.F_INVALID
    _, fl = run([C(69.0), OP(S.EXP)], z)           # e^69 ~ 9.25e29
    assert fl & oracle.F_INVALID == 0
    _, fl = run([C(69.1), OP(S.EXP)], z)           # e^69.1 ~ 1.02e30
    assert fl & oracle.F_INVALID
    # A leaf above the limit is invalid too: fp32 1e30 is 1.0000000150e30 > 1e30 in FP64.
    _, fl = run([C(1e30)], z)
    assert fl & oracle.F_INVALID


def test_validity_threshold_fp32_reads_limit_in_fp32():
    z = np.zeros((1, 1), np.float32)
    _, fl = run([C(1e30)], z, "fp32")              # the fp32 value nearest 1e30 passes
    assert fl & oracle.F_INVALID == 0
    _, fl = run([C(1e30), C(2.0), OP(S.MUL)], z, "fp32")
    assert fl & oracle.F_INVALID


def test_nan_and_hidden_overflow_are_invalid():
    z = np.zeros((1, 1), np.float32)
    # inf - inf = NaN in fp32; the NaN is caught even though no later value shows it.
    toks = [C(100), OP(S.EXP), OP(S.DUP), OP(S.SUB)]
    _, fl = run(toks, z, "fp32")
    assert fl & oracle.F_INVALID
    # An overflowing intermediate that a later protected division hides: 1 / 1e31 -> 1e-31.
    toks = [C(1.0), C(1e16), C(1e15), OP(S.MUL), OP(S.PDIV)]
    f, fl = run(toks, z)
    assert abs(f[0]) < 1e-30 and fl & oracle.F_INVALID


def test_near_threshold_diagnostic():
    z = np.zeros((1, 1), np.float32)
    _, fl = run([C(1.0), C(0.001), OP(S.PDIV)], z)
    assert fl & oracle.F_NEAR
    _, fl = run([C(1.0), C(0.5), OP(S.PDIV)], z)
    assert fl & oracle.F_NEAR == 0


# ------------------------------------------------------------------ structure
def test_structural_check():
    chk = oracle.check_program
    assert chk([S.CONST], 1) == 0
    assert chk([S.ADD], 1) == 1                      # underflow
    assert chk([S.CONST, S.CONST], 1) == 3           # two values left
    assert chk([S.LOAD0 + 2], 2) == 5                # x2 with d = 2
    assert chk([200], 1) == 4                        # unknown opcode
    assert chk([], 1) == 6
    assert chk([S.CONST] * 33 + [S.ADD] * 32, 1) == 2   # 33 values > StackSize 32
    assert chk([S.CONST] * 32 + [S.ADD] * 31, 1) == 0
    assert chk([S.CONST, S.DUP, S.SWAP, S.DEL], 1) == 0


# ------------------------------------------------------------------ paper's genomes
def _quadratic_data(n=512, seed=7):
    rng = np.random.default_rng(seed)
    a = rng.uniform(0.2, 3.0, n) * rng.choice([-1, 1], n)
    c = rng.uniform(-3.0, 3.0, n)
    b = rng.uniform(-6.0, 6.0, n)
    X = np.stack([a, b, c]).astype(np.float32)
    A, B, Cc = (X[i].astype(np.float64) for i in range(3))
    keep = B * B - 4 * A * Cc >= 0
    return X[:, keep]


@pytest.mark.parametrize("name", ["genome1", "genome2"])
def test_paper_genomes_solve_the_quadratic(name):
    """"Understanding Beagle Output": both printed genomes reach ASR 1.0 on QuadraticEq, i.e. they compute
    the root (-b + sqrt(b^2 - 4ac)) / (2a). Checked against that closed form."""
    n, toks = paper_genomes()[name]
    assert len(toks) == n
    X = _quadratic_data()
    A, B, Cc = (X[i].astype(np.float64) for i in range(3))
    root = (-B + np.sqrt(B * B - 4 * A * Cc)) / (2 * A)
    scale = (np.abs(B) + np.sqrt(B * B + 4 * np.abs(A * Cc))) / np.abs(2 * A)
    f, fl = run(toks, X)
    assert fl & oracle.F_INVALID == 0
    assert np.all(np.abs(f - root) <= 1e-13 * scale)
    f32, fl32 = run(toks, X, "fp32")
    assert np.all(np.abs(f32 - root) <= 1e-5 * scale)
    mse, omr2, _ = oracle.aggregate(f, root.astype(np.float32))
    assert omr2 < 1e-12 and mse < 1e-10


def test_paper_genome_depths():
    g = paper_genomes()
    assert S.max_depth([t[0] for t in g["genome1"][1]]) == 3
    for _, toks in g.values():
        assert oracle.check_program([t[0] for t in toks], 3) == 0


# ------------------------------------------------------------------ closed forms
def test_mse_closed_form():
    X = np.array([[1, 2, 3]], np.float32)
    prog = [LD(0), LD(0), OP(S.MUL)]
    f, fl = run(prog, X)
    mse, omr2, _ = oracle.aggregate(f, np.zeros(3, np.float32), fl)
    assert mse == 98.0 / 3.0                                  # (1 + 16 + 81) / 3
    mse, omr2, _ = oracle.aggregate(f, np.array([1, 4, 9], np.float32), fl)
    assert mse == 0.0 and omr2 == 0.0
    # y = [2, 4, 6]: residuals -1, 0, 3 -> MSE 10/3; r of (1,4,9) vs (2,4,6) by hand:
    # centred f = (-11/3, -2/3, 13/3), centred y = (-2, 0, 2): Sfy = 16, Sff = 98/3, Syy = 8,
    # so r^2 = 16^2 / (98/3 * 8) = 48/49 and 1 - r^2 = 1/49.
    mse, omr2, _ = oracle.aggregate(f, np.array([2, 4, 6], np.float32), fl)
    assert mse == pytest.approx(10.0 / 3.0, rel=1e-15)
    assert omr2 == pytest.approx(1.0 / 49.0, rel=1e-13)


def test_c1_target_program_has_rounding_level_mse():
    pr = S.make_c1(P=1)
    toks = S.C1_TARGET_PROGRAM
    f, fl = run(toks, pr.X)
    exact = S.c1_target(pr.X)
    assert np.all(np.abs(f - exact) <= 1e-14 * (np.abs(exact) + 1))
    half_ulp = np.spacing(np.abs(pr.y)).astype(np.float64) / 2
    mse, omr2, _ = oracle.aggregate(f, pr.y, fl)
    bound = np.mean((half_ulp + 1e-14 * (np.abs(exact) + 1)) ** 2)
    assert 0.0 <= mse <= bound
    assert 0.0 <= omr2 < 1e-12


def test_one_minus_r2_matches_numpy_and_least_squares():
    rng = np.random.default_rng(3)
    for _ in range(20):
        X = rng.uniform(-3, 3, size=(2, 257)).astype(np.float32)
        y = (rng.normal(size=257) + X[0]).astype(np.float32)
        progs = S.gen_programs(rng, 1, 5, 20, 2)
        f, fl = oracle.eval_program(progs.ops, progs.consts, X)
        if fl & oracle.F_INVALID or np.all(f == f[0]):
            continue
        _, omr2, _ = oracle.aggregate(f, y, fl)
        r = np.corrcoef(f, y.astype(np.float64))[0, 1]
        assert omr2 == pytest.approx(1 - r * r, rel=1e-10, abs=1e-13)
        # 1 - r^2 is the residual of the best affine fit y ~ alpha + beta f over S_yy.
        A = np.stack([np.ones_like(f), f], 1)
        yd = y.astype(np.float64)
        coef = np.linalg.lstsq(A, yd, rcond=None)[0]
        res = np.sum((yd - A @ coef) ** 2) / np.sum((yd - yd.mean()) ** 2)
        assert omr2 == pytest.approx(res, rel=1e-8, abs=1e-12)


def test_affine_transform_of_target_has_zero_one_minus_r2():
    pr = S.make_c1(P=1)
    toks = [C(1.25)] + S.C1_TARGET_PROGRAM + [C(-0.75), OP(S.MUL), OP(S.ADD)]
    f, fl = run(toks, pr.X)
    yexact = S.c1_target(pr.X)
    _, omr2, _ = oracle.aggregate(f, yexact.astype(np.float32), fl)
    assert omr2 < 1e-12


def test_degenerate_when_output_is_constant():
    X = np.array([[1, 2, 3]], np.float32)
    y = np.array([1, 0, 2], np.float32)
    for toks in ([C(1.5)], [LD(0), LD(0), OP(S.SUB)]):
        f, fl = run(toks, X)
        mse, omr2, fl2 = oracle.aggregate(f, y, fl)
        assert fl2 & oracle.F_DEGENERATE and omr2 == 1.0
        assert mse == pytest.approx(np.mean((f - y.astype(np.float64)) ** 2))


def test_invalid_program_scores_infinity():
    X = np.array([[1, 2, 3]], np.float32)
    f, fl = run([C(100.0), OP(S.EXP)], X)
    mse, omr2, fl2 = oracle.aggregate(f, np.zeros(3, np.float32), fl)
    assert fl2 & oracle.F_INVALID and mse == math.inf and omr2 == math.inf


# ------------------------------------------------------------------ invariants
def test_permutation_invariance():
    pr = S.make_c1(P=64, N=300)
    perm = np.random.default_rng(0).permutation(pr.N)
    a = oracle.score_programs(pr.programs, pr.X, pr.y)
    b = oracle.score_programs(pr.programs, pr.X[:, perm], pr.y[perm])
    assert np.array_equal(a[2], b[2])
    ok = np.isfinite(a[0])
    np.testing.assert_allclose(a[0][ok], b[0][ok], rtol=1e-14)
    np.testing.assert_allclose(a[1][ok], b[1][ok], rtol=1e-10, atol=1e-14)


def test_population_score_equals_per_program_eval():
    pr = S.make_c1(P=40, N=200)
    mse, omr2, flags = oracle.score_programs(pr.programs, pr.X, pr.y, nthreads=3)
    for p in range(pr.programs.P):
        ops, cs = pr.programs.program(p)
        f, fl = oracle.eval_program(ops, cs, pr.X)
        m, o, fl2 = oracle.aggregate(f, pr.y, fl)
        assert flags[p] == fl2
        assert (mse[p] == m or (math.isinf(m) and math.isinf(mse[p])))


# ------------------------------------------------------------------ brute force
_LEAVES = [LD(0), LD(1), C(0.5), C(-2.0), C(1e20)]
_UNARY = [OP(o) for o in S.UNARY]
_BINARY = [OP(o) for o in S.BINARY]


def _all_programs(max_len):
    """Every valid program up to max_len tokens over the alphabet above."""
    out = []

    def rec(seq, depth):
        if depth == 1 and seq:
            out.append(list(seq))
        if len(seq) == max_len:
            return
        remaining = max_len - len(seq)
        for t in _LEAVES:
            if depth <= remaining - 1:
                rec(seq + [t], depth + 1)
        if depth >= 1:
            for t in _UNARY:
                rec(seq + [t], depth)
        if depth >= 2:
            for t in _BINARY:
                rec(seq + [t], depth - 1)
    rec([], 0)
    return out


def _tree(tokens):
    """Rebuild the expression tree from the end of the token list (no stack machine)."""
    def parse(pos):
        op, c = tokens[pos]
        if op == S.CONST or op >= S.LOAD0:
            return (op, c), pos - 1
        if op in S.UNARY:
            child, nxt = parse(pos - 1)
            return (op, child), nxt
        right, nxt = parse(pos - 1)
        left, nxt = parse(nxt)
        return (op, left, right), nxt
    node, nxt = parse(len(tokens) - 1)
    assert nxt == -1
    return node


def _tree_eval(node, x, fp32):
    """Evaluate a tree on one case; returns (value, invalid). Rounds each op like the
    oracle's mode; the rule and protections are restated from the reading."""
    rnd = (lambda v: float(np.float32(v))) if fp32 else (lambda v: v)
    big = float(np.float32(1e30)) if fp32 else 1e30
    tiny = float(np.float32(1e-3)) if fp32 else 1e-3
    op = node[0]
    if op == S.CONST:
        v = float(np.float32(node[1]))
        return v, not (abs(v) <= big)
    if op >= S.LOAD0:
        v = float(x[op - S.LOAD0])
        return v, not (abs(v) <= big)
    if op in S.UNARY:
        a, bad = _tree_eval(node[1], x, fp32)
        try:
            v = {S.SIN: lambda: math.sin(a), S.COS: lambda: math.cos(a),
                 S.EXP: lambda: math.exp(a),
                 S.PLOG: lambda: math.log(abs(a)) if abs(a) > tiny else 0.0,
                 S.PSQRT: lambda: math.sqrt(abs(a)), S.SQUARE: lambda: a * a}[op]()
        except (OverflowError, ValueError):
            v = math.inf if op in (S.EXP, S.SQUARE) else math.nan
        v = rnd(v) if math.isfinite(v) else v
        return v, bad or not (abs(v) <= big)
    a, bad1 = _tree_eval(node[1], x, fp32)
    b, bad2 = _tree_eval(node[2], x, fp32)
    if op == S.ADD:
        v = a + b
    elif op == S.SUB:
        v = a - b
    elif op == S.MUL:
        v = a * b
    else:
        v = a / b if abs(b) > tiny else 1.0
    v = rnd(v) if math.isfinite(v) else v
    return v, bad1 or bad2 or not (abs(v) <= big)


@pytest.mark.parametrize("mode", ["fp64", "fp32"])
def test_bruteforce_all_programs_to_length_4(mode):
    X = np.array([[0.25, -1.5, 2.0, 3.0], [1.0, 0.5, -2.5, 0.0]], np.float32)
    progs = _all_programs(4)
    assert len(progs) > 1000
    for toks in progs:
        f, fl = run(toks, X, mode)
        tree = _tree(toks)
        bad_any = False
        for i in range(X.shape[1]):
            v, bad = _tree_eval(tree, X[:, i], mode == "fp32")
            bad_any |= bad
            if not bad:
                assert f[i] == v, (toks, i, f[i], v)
        assert bool(fl & oracle.F_INVALID) == bad_any, toks


def test_bruteforce_length_5_rational_ops_exact():
    """Over + - * square on dyadic data every result is exact in double, so the oracle
    must equal exact rational arithmetic on the rebuilt tree."""
    global _LEAVES, _UNARY, _BINARY
    saved = (_LEAVES, _UNARY, _BINARY)
    try:
        _LEAVES = [LD(0), LD(1), C(0.5), C(-2.0)]
        _UNARY = [OP(S.SQUARE)]
        _BINARY = [OP(S.ADD), OP(S.SUB), OP(S.MUL)]
        progs = _all_programs(5)
    finally:
        _LEAVES, _UNARY, _BINARY = saved
    X = np.array([[0.25, -1.5, 3.0], [1.0, 0.5, -2.5]], np.float32)

    def exact(node, x):
        op = node[0]
        if op == S.CONST:
            return Fraction(float(node[1]))
        if op >= S.LOAD0:
            return Fraction(float(x[op - S.LOAD0]))
        if op == S.SQUARE:
            a = exact(node[1], x)
            return a * a
        a, b = exact(node[1], x), exact(node[2], x)
        return a + b if op == S.ADD else a - b if op == S.SUB else a * b

    for toks in progs:
        f, fl = run(toks, X)
        tree = _tree(toks)
        for i in range(X.shape[1]):
            assert Fraction(f[i]) == exact(tree, X[:, i]), toks


def test_fp32_mode_matches_numpy_float32_on_ieee_ops():
    """+ - * / sqrt are IEEE-exact in fp32; numpy float32 arithmetic gives the same bits."""
    rng = np.random.default_rng(11)
    X = rng.uniform(-3, 3, size=(3, 64)).astype(np.float32)
    progs = S.gen_programs(rng, 200, 5, 40, 3, unary=(S.SQUARE, S.PSQRT),
                           binary=S.BINARY)
    for p in range(progs.P):
        ops, cs = progs.program(p)
        f, fl = oracle.eval_program(ops, cs, X, "fp32")
        st = []
        t = np.float32(1e-3)
        for op, c in zip(ops, cs):
            op = int(op)
            if op >= S.LOAD0:
                st.append(X[op - S.LOAD0].copy())
            elif op == S.CONST:
                st.append(np.full(64, c, np.float32))
            elif op == S.SQUARE:
                st.append(st.pop() ** 2)
            elif op == S.PSQRT:
                st.append(np.sqrt(np.abs(st.pop())))
            else:
                b, a = st.pop(), st.pop()
                with np.errstate(all="ignore"):
                    st.append(a + b if op == S.ADD else a - b if op == S.SUB else a * b
                              if op == S.MUL else np.where(np.abs(b) > t, a / b,
                                                           np.float32(1)))
        ref = st[0]
        if fl & oracle.F_INVALID:
            continue
        assert np.array_equal(f.astype(np.float32), ref), p
