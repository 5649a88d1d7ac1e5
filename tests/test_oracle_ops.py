"""Pins of the oracle's versions of the rest of Table 3 (POW, SIGN, CUBE, CBRT, TAN, ARCSIN,
ARCCOS, ARCTAN, TANH, COPY/PASTE): values by hand and from Python's math module, a brute
force over every short program against a tree evaluator written here, the structural rules
of COPY/PASTE, and the running error bound under perturbations within the ulp limits."""
from __future__ import annotations

import math

import numpy as np
import pytest

import oracle
from paper_2607_06731_gb300 import synth as S

X1 = np.array([[0.5, -0.25, 2.0, -8.0, 0.0]], np.float32)


def run(tokens, X=X1, mode="fp64"):
    progs = S.from_token_lists([tokens])
    ops, cs = progs.program(0)
    return oracle.eval_program(ops, cs, X, mode)


def C(v):
    return (S.CONST, float(v))


def LD(k):
    return (S.LOAD0 + k, 0.0)


def OP(o):
    return (o, 0.0)


@pytest.mark.parametrize("mode", ["fp64", "fp32"])
def test_new_opcodes_by_hand(mode):
    # POW is second ^ top
    f, fl = run([C(2), C(3), OP(S.POW)], mode=mode)
    assert np.all(f == 8.0) and fl == 0
    f, _ = run([C(4), C(0.5), OP(S.POW)], mode=mode)
    assert np.all(f == 2.0)
    f, _ = run([C(2), C(-2), OP(S.POW)], mode=mode)
    assert np.all(f == 0.25)
    _, fl = run([C(-8), C(1 / 3), OP(S.POW)], mode=mode)     # negative base, non-integer
    assert fl & oracle.F_INVALID
    _, fl = run([C(0), C(-1), OP(S.POW)], mode=mode)         # 0^-1 = inf
    assert fl & oracle.F_INVALID
    f, _ = run([C(-2), C(3), OP(S.POW)], mode=mode)          # integer power of a negative
    assert np.all(f == -8.0)
    f, _ = run([LD(0), OP(S.SIGN)], mode=mode)
    assert np.array_equal(f, -X1[0].astype(np.float64))
    f, _ = run([LD(0), OP(S.CUBE)], mode=mode)
    assert np.array_equal(f, [0.125, -0.015625, 8.0, -512.0, 0.0])
    f, _ = run([C(-27), OP(S.CBRT)], mode=mode)      # libm's cube root: within 1 ulp
    assert np.all(np.abs(f + 3.0) <= np.spacing(3.0))
    f, _ = run([C(0.5), OP(S.ASIN)], mode=mode)
    assert f[0] == pytest.approx(math.pi / 6, rel=1e-7 if mode == "fp32" else 1e-15)
    f, _ = run([C(-1), OP(S.ACOS)], mode=mode)
    assert f[0] == pytest.approx(math.pi, rel=1e-7 if mode == "fp32" else 1e-15)
    _, fl = run([C(1.5), OP(S.ASIN)], mode=mode)             # outside [-1, 1]: NaN
    assert fl & oracle.F_INVALID
    _, fl = run([C(-1.0001), OP(S.ACOS)], mode=mode)
    assert fl & oracle.F_INVALID
    f, _ = run([C(1), OP(S.ATAN)], mode=mode)
    assert f[0] == pytest.approx(math.pi / 4, rel=1e-7 if mode == "fp32" else 1e-15)
    f, _ = run([C(0.5), OP(S.TANH)], mode=mode)
    assert f[0] == pytest.approx(math.tanh(0.5), rel=1e-7 if mode == "fp32" else 1e-15)
    f, _ = run([C(0.75), OP(S.TAN)], mode=mode)
    assert f[0] == pytest.approx(math.tan(np.float32(0.75)), rel=1e-7 if mode == "fp32" else 1e-15)
    _, fl = run([C(3e10), C(2), OP(S.POW)], mode=mode)       # 9e20: valid
    assert not fl & oracle.F_INVALID
    _, fl = run([C(3e10), C(3), OP(S.POW)], mode=mode)       # 2.7e31 > 1e30: invalid
    assert fl & oracle.F_INVALID


def test_cube_rounds_twice_in_fp32():
    """CUBE is (a a) a with each product rounded to fp32, as numpy float32 computes it."""
    rng = np.random.default_rng(4)
    X = rng.uniform(-50, 50, (1, 500)).astype(np.float32)
    f, _ = run([LD(0), OP(S.CUBE)], X, "fp32")
    x = X[0]
    assert np.array_equal(f.astype(np.float32), (x * x) * x)


def test_copy_paste_semantics():
    """x0 COPY@0 x1 ADD PASTE@0 MUL = (x0 + x1) x0: COPY leaves the stack alone, PASTE
    pushes the copied value."""
    X = np.array([[1.5, -2.0, 3.0], [0.5, 4.0, -1.0]], np.float32)
    toks = [LD(0), (S.COPY0, 0.0), LD(1), OP(S.ADD), (S.PASTE0, 0.0), OP(S.MUL)]
    f, fl = run(toks, X)
    x0, x1 = X[0].astype(np.float64), X[1].astype(np.float64)
    assert fl == 0 and np.array_equal(f, (x0 + x1) * x0)
    # two variables, pasted in the other order
    toks = [LD(0), (S.COPY0 + 3, 0.0), LD(1), (S.COPY0 + 5, 0.0), OP(S.SUB),
            (S.PASTE0 + 3, 0.0), OP(S.MUL), (S.PASTE0 + 5, 0.0), OP(S.ADD)]
    f, _ = run(toks, X)
    assert np.array_equal(f, (x0 - x1) * x0 + x1)


def test_copy_paste_structure():
    chk = lambda toks: oracle.check_program(  # noqa: E731
        np.array([t[0] for t in toks], np.uint8), d=2)
    assert chk([LD(0), (S.COPY0, 0.0), (S.PASTE0, 0.0), OP(S.ADD)]) == 0
    assert chk([LD(0), (S.PASTE0, 0.0), OP(S.ADD)]) == 7                 # paste before copy
    assert chk([LD(0), (S.COPY0, 0.0), (S.COPY0, 0.0), (S.PASTE0, 0.0),
                OP(S.ADD)]) == 7                                           # copy twice
    assert chk([LD(0), (S.COPY0, 0.0)]) == 7                               # never pasted
    assert chk([(S.COPY0, 0.0), LD(0)]) == 1                               # nothing to copy
    assert chk([LD(0), (S.COPY0 + 8, 0.0)]) == 4                           # @8 does not exist
    assert chk([LD(0), (S.COPY0, 0.0), (S.PASTE0, 0.0), OP(S.ADD), (S.COPY0, 0.0),
                (S.PASTE0, 0.0), OP(S.MUL)]) == 0                          # reused after paste


# ------------------------------------------------------------------ brute force
_LEAVES = [LD(0), C(0.5), C(-2.0)]
_UNARY = [OP(o) for o in S.UNARY_EXT]
_BINARY = [OP(S.POW), OP(S.ADD)]


def _all_programs(max_len):
    out = []

    def rec(seq, depth):
        if seq and depth == 1:
            out.append(list(seq))
        if len(seq) == max_len:
            return
        left = max_len - len(seq)
        for t in _LEAVES:
            if depth + 1 - 1 <= left - 1:
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
    st = []
    for t in tokens:
        if t[0] == S.CONST or t[0] >= S.LOAD0:
            st.append((t[0], t[1]))
        elif t[0] in S.ALL_UNARY:
            st.append((t[0], st.pop()))
        else:
            b = st.pop()
            st.append((t[0], st.pop(), b))
    assert len(st) == 1
    return st[0]


def _eval(node, x, fp32):
    """Value and invalid marker of a tree on one case, each operation rounded as the mode
    rounds it; the functions are Python's math module."""
    rnd = (lambda v: float(np.float32(v))) if fp32 else (lambda v: v)
    big = float(np.float32(1e30)) if fp32 else 1e30
    op = node[0]
    if op == S.CONST:
        v = float(np.float32(node[1]))
        return v, False
    if op >= S.LOAD0:
        return float(x[op - S.LOAD0]), False
    if op in S.ALL_UNARY:
        a, bad = _eval(node[1], x, fp32)
        if not math.isfinite(a):
            return math.nan, True
        try:
            if op == S.CUBE:
                v = rnd(a * a) * a
            else:
                v = {S.SIGN: lambda: -a, S.CBRT: lambda: math.copysign(abs(a) ** (1 / 3), a)
                     if a != 0 else 0.0, S.TAN: lambda: math.tan(a),
                     S.ASIN: lambda: math.asin(a), S.ACOS: lambda: math.acos(a),
                     S.ATAN: lambda: math.atan(a), S.TANH: lambda: math.tanh(a)}[op]()
        except (OverflowError, ValueError):
            v = math.nan
        v = rnd(v) if math.isfinite(v) else v
        return v, bad or not (abs(v) <= big)
    a, b1 = _eval(node[1], x, fp32)
    b, b2 = _eval(node[2], x, fp32)
    if op == S.ADD:
        v = a + b
    else:
        try:
            v = math.pow(a, b)
        except (OverflowError, ValueError, ZeroDivisionError):
            v = math.inf if a == 0 else math.nan
    v = rnd(v) if math.isfinite(v) else v
    return v, b1 or b2 or not (abs(v) <= big)


@pytest.mark.parametrize("mode", ["fp64", "fp32"])
def test_bruteforce_new_ops_to_length_4(mode):
    X = np.array([[0.25, -0.75, 1.5, 3.0]], np.float32)
    progs = _all_programs(4)
    assert len(progs) > 500
    for toks in progs:
        f, fl = run(toks, X, mode)
        tree = _tree(toks)
        bad_any = False
        for i in range(X.shape[1]):
            v, bad = _eval(tree, X[:, i], mode == "fp32")
            bad_any |= bad
            if bad:
                continue
            if any(t[0] == S.CBRT for t in toks):
                # Python's cube root is a power: compare within an ulp of the result
                assert f[i] == pytest.approx(v, rel=3e-16 if mode == "fp64" else 1.2e-7), toks
            else:
                assert f[i] == v, (toks, i, f[i], v)
        assert bool(fl & oracle.F_INVALID) == bad_any, toks


def test_copy_paste_brute_force_against_inlining():
    """A program with COPY@0 ... PASTE@0 equals the same program with the copied subexpression
    written out again at the paste (register-free), on every case."""
    rng = np.random.default_rng(9)
    X = rng.uniform(-2, 2, (2, 40)).astype(np.float32)
    base = S.gen_programs(rng, 300, 3, 20, 2, unary=S.UNARY + S.UNARY_EXT,
                          binary=S.ALL_BINARY)
    withr = S.with_registers(base, rng, frac=1.0, n_regs=1)
    for p in range(withr.P):
        ops, cs = withr.program(p)
        toks = [(int(o), float(c)) for o, c in zip(ops, cs)]
        # inline: the value copied is the subtree ending at the token before COPY
        i = next(k for k, t in enumerate(toks) if t[0] == S.COPY0)
        j = next(k for k, t in enumerate(toks) if t[0] == S.PASTE0)
        depth, start = 0, i
        for k in range(i, -1, -1):        # find where that subtree starts
            need, delta = S.stack_effect(toks[k][0])
            depth += delta
            if depth == 1:
                start = k
                break
        sub = toks[start:i + 1]
        inl = toks[:i] + toks[i:i + 1] + toks[i + 1:j] + sub + toks[j + 1:]
        inl = [t for t in inl if t[0] != S.COPY0]
        f1, fl1 = oracle.eval_program(ops, cs, X, "fp64")
        pr2 = S.from_token_lists([inl])
        f2, fl2 = oracle.eval_program(*pr2.program(0), X, "fp64")
        assert fl1 & oracle.F_MALFORMED == 0
        assert (fl1 & 1) == (fl2 & 1)
        if not fl1 & 1:
            assert np.array_equal(f1, f2), p


def test_bound_holds_for_new_ops():
    """Perturb every transcendental result of the new ops within its ulp limit (in a
    re-implementation of the evaluation here) and check that the outputs stay within the
    oracle's per-case bound."""
    rng = np.random.default_rng(12)
    X = rng.uniform(-1.5, 1.5, (2, 64)).astype(np.float32)
    progs = S.gen_programs(rng, 150, 3, 16, 2, unary=S.UNARY_EXT + (S.SQUARE,),
                           binary=(S.ADD, S.MUL, S.POW))
    lim = oracle.DEV_ULPS_FP64
    fns = {S.CBRT: np.cbrt, S.TAN: np.tan, S.ASIN: np.arcsin, S.ACOS: np.arccos,
           S.ATAN: np.arctan, S.TANH: np.tanh}
    for p in range(progs.P):
        ops, cs = progs.program(p)
        f, dl, fl = oracle.eval_bound(ops, cs, X, "fp64")
        if fl & (oracle.F_INVALID | oracle.F_AMBIG | oracle.F_MALFORMED):
            continue
        for trial in range(4):
            st = []
            with np.errstate(all="ignore"):
                for op, c in zip(ops, cs):
                    op = int(op)
                    if op >= S.LOAD0:
                        st.append(X[op - S.LOAD0].astype(np.float64))
                    elif op == S.CONST:
                        st.append(np.full(64, float(c)))
                    elif op in fns or op == S.POW:
                        if op == S.POW:
                            b, a = st.pop(), st.pop()
                            v = np.power(a, b)
                        else:
                            v = fns[op](st.pop())
                        # numpy's own result is within 1 ulp of the exact value, so
                        # perturbing it by (limit - 1) ulps keeps the simulated device
                        # within its limit of the exact value
                        u = rng.uniform(-(lim[op] - 1), lim[op] - 1, 64)
                        st.append(v + u * np.spacing(np.abs(v)))
                    elif op == S.SIGN:
                        st.append(-st.pop())
                    elif op == S.CUBE:
                        a = st.pop()
                        st.append((a * a) * a)
                    elif op == S.SQUARE:
                        a = st.pop()
                        st.append(a * a)
                    else:
                        b, a = st.pop(), st.pop()
                        st.append(a + b if op == S.ADD else a * b)
            assert np.all(np.abs(st[0] - f) <= dl * 1.0000001 + 1e-300), p
