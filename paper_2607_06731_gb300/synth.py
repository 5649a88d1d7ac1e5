"""Seeded synthetic inputs for population scoring: random postfix programs and datasets.

This module only draws inputs. It scores nothing: it computes no fitness, applies no
protected operator and checks no intermediate value. The CUDA path and the oracle both
consume what it returns and share nothing else.

Programs are Beagle GCL genomes (the GCL section, Table 3): postfix token lists run on a value
stack. The paper draws new genomes by mutation on the CPU ("Dividing Tasks Between CPU and GPU"); this generator
stands in for that host side with a plain random walk over valid programs. Datasets stand
in for a user's ``MLSetup.GetNextInputsAndCorrectOutput`` data source (the MLSetup mandatory overrides): each
config draws inputs X and computes a target y from a fixed or random expression.

Wire format (one byte per token; must match ``include/beagle.h``):

    0 CONST   1 ADD   2 SUB   3 MUL   4 PDIV   5 SIN   6 COS   7 EXP   8 PLOG
    9 PSQRT  10 SQUARE  11 DUP  12 SWAP  13 DEL  14 POW  15 SIGN  16 CUBE  17 CBRT
   18 TAN   19 ASIN  20 ACOS  21 ATAN  22 TANH   32+k LOAD x_k (k < 16)
   64+k COPY @k   80+k PASTE @k (k < 8)

``consts`` is token-aligned: ``consts[offsets[p] + j]`` is the value of token j of program
p when that token is CONST (fp32), and 0 otherwise.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

CONST, ADD, SUB, MUL, PDIV = 0, 1, 2, 3, 4
SIN, COS, EXP, PLOG, PSQRT, SQUARE = 5, 6, 7, 8, 9, 10
DUP, SWAP, DEL = 11, 12, 13
POW, SIGN, CUBE, CBRT, TAN, ASIN, ACOS, ATAN, TANH = 14, 15, 16, 17, 18, 19, 20, 21, 22
LOAD0 = 32
COPY0, PASTE0, N_REGS = 64, 80, 8
MAX_VARS = 16

# The default operator set of the benchmark workloads, and the rest of Table 3.
UNARY = (SIN, COS, EXP, PLOG, PSQRT, SQUARE)
BINARY = (ADD, SUB, MUL, PDIV)
UNARY_EXT = (SIGN, CUBE, CBRT, TAN, ASIN, ACOS, ATAN, TANH)
ALL_UNARY = UNARY + UNARY_EXT
ALL_BINARY = BINARY + (POW,)
NAMES = {CONST: "CONST", ADD: "ADD", SUB: "SUB", MUL: "MUL", PDIV: "PDIV", SIN: "SIN",
         COS: "COS", EXP: "EXP", PLOG: "PLOG", PSQRT: "PSQRT", SQUARE: "SQUARE",
         DUP: "DUP", SWAP: "SWAP", DEL: "DEL", POW: "POW", SIGN: "SIGN", CUBE: "CUBE",
         CBRT: "CBRT", TAN: "TAN", ASIN: "ARCSIN", ACOS: "ARCCOS", ATAN: "ARCTAN",
         TANH: "TANH"}


def allowed_operations(exclude=()):
    """The generator's operator sets without the excluded opcodes: the analogue of
    MLSetup.GetAllowedOperations ("Subclassing MLSetup - optional overrides"), which restricts
    the operators evolution may use. Returns (unary, binary) for gen_programs."""
    ex = set(exclude)
    return (tuple(o for o in ALL_UNARY if o not in ex),
            tuple(o for o in ALL_BINARY if o not in ex))

# Class weights of the random walk: leaf / unary / binary, renormalised over the classes
# that can still end in a depth-1 program. The paper gives no distribution; this is ours.
CLASS_WEIGHTS = (0.40, 0.25, 0.35)
DEFAULT_DEPTH_CAP = 16


@dataclasses.dataclass
class Programs:
    """A population in the wire format (concatenated tokens + per-program offsets)."""
    ops: np.ndarray        # uint8 [T]
    offsets: np.ndarray    # int64 [P]
    lengths: np.ndarray    # int32 [P]
    consts: np.ndarray     # float32 [T], token-aligned

    @property
    def P(self) -> int:
        return int(self.lengths.shape[0])

    @property
    def tokens(self) -> int:
        return int(self.ops.shape[0])

    def program(self, p: int):
        o, n = int(self.offsets[p]), int(self.lengths[p])
        return self.ops[o:o + n], self.consts[o:o + n]

    def subset(self, idx) -> "Programs":
        idx = np.asarray(idx, dtype=np.int64)
        lens = self.lengths[idx]
        offs = np.zeros(len(idx), np.int64)
        if len(idx) > 1:
            offs[1:] = np.cumsum(lens[:-1], dtype=np.int64)
        gather = (np.repeat(self.offsets[idx] - offs, lens) +
                  np.arange(int(lens.sum()), dtype=np.int64))
        return Programs(self.ops[gather].copy(), offs, lens.astype(np.int32),
                        self.consts[gather].copy())


def _rng(seed) -> np.random.Generator:
    if isinstance(seed, np.random.Generator):
        return seed
    return np.random.Generator(np.random.PCG64(np.random.SeedSequence(seed)))


def from_token_lists(progs) -> Programs:
    """Pack a list of programs given as lists of (opcode, const) pairs."""
    lens = np.array([len(p) for p in progs], np.int32)
    offs = np.zeros(len(progs), np.int64)
    if len(progs) > 1:
        offs[1:] = np.cumsum(lens[:-1], dtype=np.int64)
    ops = np.array([t[0] for p in progs for t in p], np.uint8)
    cs = np.array([t[1] for p in progs for t in p], np.float32)
    return Programs(ops, offs, lens, cs)


def gen_programs(seed, P: int, lmin: int, lmax: int, d: int, *,
                 depth_cap: int = DEFAULT_DEPTH_CAP, weights=CLASS_WEIGHTS,
                 unary=UNARY, binary=BINARY, const_lo: float = -2.0,
                 const_hi: float = 2.0, p_var: float = 0.5,
                 lengths: np.ndarray | None = None) -> Programs:
    """Draw P valid postfix programs with lengths uniform in [lmin, lmax].

    Token-by-token random walk over all programs at once. With s values on the stack and
    r tokens left (this one included) a class is feasible when the program can still end at
    depth exactly 1 without passing ``depth_cap``:
      leaf   s + 1 <= depth_cap and s <= r - 1
      unary  s >= 1 and s - 1 <= r - 1
      binary s >= 2 and s - 2 <= r - 1
    Leaves are a variable x_k (k uniform below d) with probability p_var, else an fp32
    constant uniform in [const_lo, const_hi]. Ops are uniform within their class.
    """
    rng = _rng(seed)
    if lengths is None:
        L = rng.integers(lmin, lmax + 1, size=P).astype(np.int32)
    else:
        L = np.asarray(lengths, np.int32)
        P = len(L)
    if P and int(L.min()) < 1:
        raise ValueError("program length must be >= 1")
    offs = np.zeros(P, np.int64)
    if P > 1:
        offs[1:] = np.cumsum(L[:-1], dtype=np.int64)
    total = int(L.sum()) if P else 0
    ops = np.zeros(total, np.uint8)
    consts = np.zeros(total, np.float32)
    s = np.zeros(P, np.int32)
    unary = np.asarray(unary, np.uint8)
    binary = np.asarray(binary, np.uint8)
    w_leaf, w_un, w_bin = weights
    if len(unary) == 0:
        w_un = 0.0
    lmax_eff = int(L.max()) if P else 0
    for t in range(lmax_eff):
        act = np.nonzero(L > t)[0]
        r = L[act] - t
        sa = s[act]
        wl = w_leaf * ((sa + 1 <= depth_cap) & (sa <= r - 1))
        wu = w_un * ((sa >= 1) & (sa - 1 <= r - 1))
        wb = w_bin * ((sa >= 2) & (sa - 2 <= r - 1))
        u = rng.random(len(act)) * (wl + wu + wb)
        cls = np.where(u < wl, 0, np.where(u < wl + wu, 1, 2))
        op = np.empty(len(act), np.uint8)
        leaf = cls == 0
        nl = int(leaf.sum())
        is_var = (rng.random(nl) < p_var) if d > 0 else np.zeros(nl, bool)
        var = rng.integers(0, max(d, 1), size=nl)
        cval = rng.uniform(const_lo, const_hi, size=nl).astype(np.float32)
        op[leaf] = np.where(is_var, LOAD0 + var, CONST).astype(np.uint8)
        pos = offs[act] + t
        consts[pos[leaf]] = np.where(is_var, np.float32(0), cval)
        un = cls == 1
        op[un] = unary[rng.integers(0, len(unary), size=int(un.sum()))] if len(unary) else 0
        bi = cls == 2
        op[bi] = binary[rng.integers(0, len(binary), size=int(bi.sum()))]
        ops[pos] = op
        s[act] = sa + np.where(leaf, 1, np.where(bi, -1, 0))
    return Programs(ops, offs, L, consts)


def stack_effect(op: int) -> tuple[int, int]:
    """(minimum depth before the token, depth change) of one token (Table 3)."""
    if op == CONST or LOAD0 <= op < LOAD0 + MAX_VARS:
        return 0, 1
    if COPY0 <= op < COPY0 + N_REGS:
        return 1, 0
    if PASTE0 <= op < PASTE0 + N_REGS:
        return 0, 1
    if op in ALL_BINARY:
        return 2, -1
    if op in ALL_UNARY:
        return 1, 0
    return {DUP: (1, 1), SWAP: (2, 0), DEL: (1, -1)}[op]


def with_registers(progs: "Programs", seed, frac: float = 0.5, n_regs: int = 2) -> "Programs":
    """Insert COPY @k / PASTE @k pairs (Table 3's variables) into a fraction of the programs:
    COPY @k after a random token, and later PASTE @k followed by ADD, so that the pasted value
    is consumed and the program still ends at depth 1. Register k is used at most once per
    program; registers 0..n_regs-1 are drawn in order."""
    rng = _rng(seed)
    out = []
    for p in range(progs.P):
        ops, cs = progs.program(p)
        toks = [(int(o), float(c)) for o, c in zip(ops, cs)]
        if rng.random() < frac and len(toks) >= 2:
            for k in range(int(rng.integers(1, n_regs + 1))):
                n = len(toks)
                i = int(rng.integers(0, n - 1))          # COPY after token i
                j = int(rng.integers(i + 1, n))          # PASTE, ADD after token j (j > i)
                toks = (toks[:i + 1] + [(COPY0 + k, 0.0)] + toks[i + 1:j + 1] +
                        [(PASTE0 + k, 0.0), (ADD, 0.0)] + toks[j + 1:])
        out.append(toks)
    return from_token_lists(out)


def max_depth(ops) -> int:
    s, m = 0, 0
    for op in ops:
        s += stack_effect(int(op))[1]
        m = max(m, s)
    return m


# ---------------------------------------------------------------------------------------
# Targets. A target is a random expression over {+, -, *, sin, cos, square}, written as a
# postfix token list and evaluated here in float64 with plain numpy math. Only these
# unprotected operators appear, so a target is defined without any protection convention.
# ---------------------------------------------------------------------------------------
TARGET_UNARY = (SIN, COS, SQUARE)
TARGET_BINARY = (ADD, SUB, MUL)


def _target_value(ops, consts, X: np.ndarray) -> np.ndarray:
    st = []
    n = X.shape[1]
    for op, c in zip(ops, consts):
        op = int(op)
        if op >= LOAD0:
            st.append(X[op - LOAD0].astype(np.float64))
        elif op == CONST:
            st.append(np.full(n, float(c)))
        elif op in TARGET_UNARY:
            a = st.pop()
            st.append(np.sin(a) if op == SIN else np.cos(a) if op == COS else a * a)
        else:
            b, a = st.pop(), st.pop()
            st.append(a + b if op == ADD else a - b if op == SUB else a * b)
    assert len(st) == 1
    return st[0]


def random_target(rng, n_nodes: int, X: np.ndarray, max_abs: float = 1e6):
    """Draw a random n-node target expression that is finite, bounded and non-constant
    on X. Returns (ops, consts, y_float64)."""
    d = X.shape[0]
    for _ in range(1000):
        t = gen_programs(rng, 1, n_nodes, n_nodes, d, unary=TARGET_UNARY,
                         binary=TARGET_BINARY, depth_cap=8)
        if not any(int(o) >= LOAD0 for o in t.ops):
            continue
        y = _target_value(t.ops, t.consts, X)
        if np.all(np.isfinite(y)) and np.max(np.abs(y)) <= max_abs and np.std(y) > 1e-3:
            return t.ops.copy(), t.consts.copy(), y
    raise RuntimeError("no admissible target expression found")


# ---------------------------------------------------------------------------------------
# Workloads
# ---------------------------------------------------------------------------------------
@dataclasses.dataclass
class Problem:
    """One population scored against one dataset."""
    name: str
    programs: Programs
    X: np.ndarray          # float32 [d][N], column-major by case (row k = variable x_k)
    y: np.ndarray          # float32 [N]
    meta: dict

    @property
    def N(self) -> int:
        return int(self.X.shape[1])

    @property
    def d(self) -> int:
        return int(self.X.shape[0])

    @property
    def node_evals(self) -> int:
        return int(self.programs.lengths.sum(dtype=np.int64)) * self.N


def c1_target(X: np.ndarray) -> np.ndarray:
    x0, x1 = X[0].astype(np.float64), X[1].astype(np.float64)
    return x0 * np.sin(x1) + 0.5 * x0 * x0


# The program equal to c1_target: x0 x1 sin * 0.5 x0 square * +
C1_TARGET_PROGRAM = [(LOAD0 + 0, 0.0), (LOAD0 + 1, 0.0), (SIN, 0.0), (MUL, 0.0),
                     (CONST, 0.5), (LOAD0 + 0, 0.0), (SQUARE, 0.0), (MUL, 0.0),
                     (ADD, 0.0)]


def _loguniform_int(rng, lo, hi, size=None):
    return np.round(np.exp(rng.uniform(math.log(lo), math.log(hi), size=size))).astype(np.int64)


def make_c1(seed: int = 1, P: int = 1024, N: int = 1024) -> Problem:
    """Plain scoring: P programs of length U{8..32} over x0, x1; N cases, X ~ U[-3, 3];
    y = x0 sin(x1) + 0.5 x0^2."""
    rng = _rng([seed, 1])
    X = rng.uniform(-3, 3, size=(2, N)).astype(np.float32)
    y = c1_target(X).astype(np.float32)
    progs = gen_programs(_rng([seed, 2]), P, 8, 32, 2)
    return Problem("c1-plain-1k", progs, X, y, {"seed": seed, "target": "x0*sin(x1)+0.5*x0^2"})


def make_c2(seed: int = 2, P: int = 100_000, N: int = 1024) -> Problem:
    """Paper-style batch: P programs of length U{16..128}, d = 5, N cases, X ~ U[-3, 3];
    y = a random 20-node expression + N(0, sigma^2 = 0.01) noise."""
    rng = _rng([seed, 1])
    d = 5
    X = rng.uniform(-3, 3, size=(d, N)).astype(np.float32)
    tops, tcs, y = random_target(rng, 20, X)
    y = (y + rng.normal(0.0, 0.1, size=N)).astype(np.float32)
    progs = gen_programs(_rng([seed, 2]), P, 16, 128, d)
    return Problem("c2-population-100k", progs, X, y,
                   {"seed": seed, "target_ops": tops, "target_consts": tcs, "noise_sigma": 0.1})


def make_c3(seed: int = 3, P: int = 50_000, N: int = 1_000_000) -> Problem:
    """Precision: P programs of length U{16..64}, d = 10, N cases, X ~ N(0, 1);
    y = a random 30-node expression scaled to RMS 1e3 + N(0, 1) noise."""
    rng = _rng([seed, 1])
    d = 10
    X = rng.standard_normal(size=(d, N)).astype(np.float32)
    tops, tcs, y = random_target(rng, 30, X, max_abs=1e8)
    y = y * (1e3 / math.sqrt(float(np.mean(y * y))))
    y = (y + rng.standard_normal(size=N)).astype(np.float32)
    progs = gen_programs(_rng([seed, 2]), P, 16, 64, d)
    return Problem("c3-precision-1m", progs, X, y,
                   {"seed": seed, "target_ops": tops, "target_consts": tcs, "rms": 1e3})


def make_c4(seed: int = 4, n_pops: int = 64, scale: float = 1.0) -> list[Problem]:
    """Ragged batching: n_pops populations, P log-uniform in [1e3, 2e5], length U{4..256},
    N log-uniform in [256, 1e5], d uniform in {1..10}, X ~ U[-5, 5]; each population has
    its own dataset with a random 10-node target + N(0, 0.01) noise. ``scale`` shrinks P and N
    (for tests) without changing the draw order."""
    rng = _rng([seed, 0])
    Ps = _loguniform_int(rng, 1_000, 200_000, n_pops)
    Ns = _loguniform_int(rng, 256, 100_000, n_pops)
    ds = rng.integers(1, 11, size=n_pops)
    out = []
    for i in range(n_pops):
        P = max(1, int(Ps[i] * scale))
        N = max(2, int(Ns[i] * scale))
        d = int(ds[i])
        r = _rng([seed, 1, i])
        X = r.uniform(-5, 5, size=(d, N)).astype(np.float32)
        tops, tcs, y = random_target(r, 10, X)
        y = (y + r.normal(0.0, 0.1, size=N)).astype(np.float32)
        progs = gen_programs(_rng([seed, 2, i]), P, 4, 256, d)
        out.append(Problem(f"c4-pop{i}", progs, X, y, {"seed": seed, "pop": i}))
    return out


def make_serving_runs(seed: int = 5, n_runs: int = 16, scale: float = 1.0):
    """Serving: n_runs evolutionary runs, each with a resident dataset (N log-uniform in
    [512, 65536], d uniform in {1..10}, X ~ U[-3, 3], a random 10-node target + noise) and a
    request generator drawing P log-uniform in [1e4, 5e5] programs of length U{8..200}."""
    rng = _rng([seed, 0])
    Ns = _loguniform_int(rng, 512, 65_536, n_runs)
    ds = rng.integers(1, 11, size=n_runs)
    runs = []
    for i in range(n_runs):
        N = max(2, int(Ns[i] * scale))
        d = int(ds[i])
        r = _rng([seed, 1, i])
        X = r.uniform(-3, 3, size=(d, N)).astype(np.float32)
        _, _, y = random_target(r, 10, X)
        y = (y + r.normal(0.0, 0.1, size=N)).astype(np.float32)
        runs.append({"run": i, "X": X, "y": y, "d": d, "N": N})
    return runs


def serving_request(seed: int, run: int, gen: int, d: int, scale: float = 1.0) -> Programs:
    r = _rng([seed, 2, run, gen])
    P = max(1, int(_loguniform_int(r, 10_000, 500_000) * scale))
    return gen_programs(r, P, 8, 200, d)


CONFIG_MAKERS = {"c1": make_c1, "c2": make_c2, "c3": make_c3}
