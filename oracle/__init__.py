"""Oracle: a plain, slow FP64 CPU scorer for Beagle population fitness.

TEST INFRASTRUCTURE ONLY. It is loaded by the tests, by the package's ``smoke()`` check and
by the benchmark's CPU-baseline leg, and by nothing on the product path. It shares no code
with the CUDA path; see ``oracle.c`` for what it computes and which passages it follows.

Pins (tests/test_oracle_*.py): the paper's two worked genomes against the closed-form
quadratic root ("Understanding Beagle Output"); per-opcode values by hand (Table 3); closed-form MSE;
1 - r^2 against numpy's correlation and a least-squares fit; invariance under permuting
cases; brute force over every program up to length 5 on a tiny alphabet against an exact
rational evaluator built on a different algorithm (tree reconstruction).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

FP64, FP32 = 0, 1
F_INVALID, F_DEGENERATE, F_MALFORMED, F_NEAR, F_AMBIG = 1, 2, 4, 256, 512
F_PERFECT = 16
# The paper's fitness functions (oracle_fit_score): correlation score of Eq. 2, the Eq. 5
# point-to-point family, and the validation test of the interactive V command.
FIT_CORRELATION, FIT_STD, FIT_STD_SQUARE, FIT_STD_CUBE, FIT_STD_HYPER, FIT_VALIDATE = range(1, 7)

# The device's per-operator accuracy (units in the last place) used in the error bounds,
# indexed by opcode. FP32 path: sin, cos, exp and the log within 2 ulp (CUDA documents 2 for
# sinf/cosf/expf; the FP32 path's own sin/cos/exp/log are tested to 2 on the GPU). FP64 path:
# CUDA's documented bounds for double sin, cos, exp, log: 2, 2, 1, 1.
DEV_ULPS_FP32 = {5: 2.0, 6: 2.0, 7: 2.0, 8: 2.0}
DEV_ULPS_FP64 = {5: 2.0, 6: 2.0, 7: 1.0, 8: 1.0}
# The rest of Table 3 (POW 14, CBRT 17, TAN 18, ARCSIN 19, ARCCOS 20, ARCTAN 21, TANH 22):
# CUDA's powf, cbrtf, tanf, asinf, acosf, atanf, tanhf and their double versions, with the
# bounds the GPU tests measure them against (tests/test_gpu_ops.py).
DEV_ULPS_FP32.update({14: 8.0, 17: 2.0, 18: 4.0, 19: 4.0, 20: 4.0, 21: 4.0, 22: 4.0})
DEV_ULPS_FP64.update({14: 2.0, 17: 2.0, 18: 2.0, 19: 2.0, 20: 2.0, 21: 2.0, 22: 2.0})
STACK = 32
CHECK_ERRORS = {0: "ok", 1: "underflow", 2: "overflow", 3: "final depth", 4: "opcode",
                5: "variable", 6: "empty", 7: "register"}

_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so (gcc, OpenMP, no fast-math, no FP contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
                               "-ffp-contract=off", "-fno-fast-math", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        P = ctypes.c_void_p
        L.oracle_check_program.argtypes = [P, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32]
        L.oracle_check_program.restype = ctypes.c_int
        L.oracle_eval.argtypes = [P, P, ctypes.c_int32, P, ctypes.c_int64, ctypes.c_int32,
                                  ctypes.c_int32, P]
        L.oracle_eval.restype = ctypes.c_uint32
        L.oracle_aggregate.argtypes = [P, P, ctypes.c_int64, ctypes.c_uint32, P, P, P]
        L.oracle_aggregate.restype = None
        L.oracle_score.argtypes = [P, P, P, P, ctypes.c_int64, P, P, ctypes.c_int64,
                                   ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, P, P, P]
        L.oracle_score.restype = ctypes.c_int
        L.oracle_threads.restype = ctypes.c_int
        L.oracle_eval_bound.argtypes = [P, P, ctypes.c_int32, P, ctypes.c_int64,
                                        ctypes.c_int32, ctypes.c_int32, P, P, P]
        L.oracle_eval_bound.restype = ctypes.c_uint32
        L.oracle_score_bound.argtypes = [P, P, P, P, ctypes.c_int64, P, P, ctypes.c_int64,
                                         ctypes.c_int32, ctypes.c_int32, P, ctypes.c_int32,
                                         P, P, P, P, P]
        L.oracle_score_bound.restype = ctypes.c_int
        L.oracle_eval_cases.argtypes = [P, P, ctypes.c_int32, P, ctypes.c_int64,
                                        ctypes.c_int32, ctypes.c_int32, P, P]
        L.oracle_eval_cases.restype = ctypes.c_uint32
        L.oracle_fit_aggregate.argtypes = [P, P, P, ctypes.c_int64, ctypes.c_uint32,
                                           ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                           ctypes.c_double, ctypes.c_int32, P, P, P]
        L.oracle_fit_aggregate.restype = None
        L.oracle_fit_score.argtypes = [P, P, P, P, ctypes.c_int64, P, P, ctypes.c_int64,
                                       ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                       ctypes.c_int32, ctypes.c_double, ctypes.c_int32, P, P, P]
        L.oracle_fit_score.restype = ctypes.c_int
        L.oracle_rank.argtypes = [P, ctypes.c_int64, P, ctypes.c_int32, P, P, P]
        L.oracle_rank.restype = ctypes.c_int
        _lib = L
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _mode(mode) -> int:
    if mode in (FP64, "fp64"):
        return FP64
    if mode in (FP32, "fp32"):
        return FP32
    raise ValueError(mode)


def threads() -> int:
    return int(lib().oracle_threads())


def check_program(ops, d: int, max_depth: int = STACK) -> int:
    ops = np.ascontiguousarray(ops, np.uint8)
    return int(lib().oracle_check_program(_p(ops), len(ops), d, max_depth))


def eval_program(ops, consts, X, mode="fp64"):
    """Outputs of one program on every case: (f float64 [N], flags)."""
    ops = np.ascontiguousarray(ops, np.uint8)
    consts = np.ascontiguousarray(consts, np.float32)
    X = np.ascontiguousarray(X, np.float32)
    if X.ndim == 1:
        X = X[None, :]
    d, N = X.shape
    f = np.zeros(N, np.float64)
    fl = lib().oracle_eval(_p(ops), _p(consts), len(ops), _p(X), N, d, _mode(mode), _p(f))
    return f, int(fl)


def aggregate(f, y, flags: int = 0):
    """(mse, one_minus_r2, flags) of given outputs f against targets y."""
    f = np.ascontiguousarray(f, np.float64)
    y = np.ascontiguousarray(y, np.float32)
    mse, omr2, fl = ctypes.c_double(), ctypes.c_double(), ctypes.c_uint32()
    lib().oracle_aggregate(_p(f), _p(y), len(y), flags, ctypes.byref(mse), ctypes.byref(omr2),
                           ctypes.byref(fl))
    return mse.value, omr2.value, fl.value


def score(ops, offsets, lengths, consts, X, y, mode="fp64", nthreads: int = 0):
    """Score a population: returns (mse [P], one_minus_r2 [P], flags [P])."""
    ops = np.ascontiguousarray(ops, np.uint8)
    offsets = np.ascontiguousarray(offsets, np.int64)
    lengths = np.ascontiguousarray(lengths, np.int32)
    consts = np.ascontiguousarray(consts, np.float32)
    X = np.ascontiguousarray(X, np.float32)
    if X.ndim == 1:
        X = X[None, :]
    y = np.ascontiguousarray(y, np.float32)
    d, N = X.shape
    P = len(lengths)
    mse = np.zeros(P, np.float64)
    omr2 = np.zeros(P, np.float64)
    flags = np.zeros(P, np.uint32)
    rc = lib().oracle_score(_p(ops), _p(offsets), _p(lengths), _p(consts), P, _p(X), _p(y), N,
                            d, _mode(mode), nthreads, _p(mse), _p(omr2), _p(flags))
    if rc != 0:
        raise ValueError("oracle_score rejected its arguments")
    return mse, omr2, flags


def score_programs(progs, X, y, mode="fp64", nthreads: int = 0):
    """Same as ``score`` for any object with ops/offsets/lengths/consts attributes."""
    return score(progs.ops, progs.offsets, progs.lengths, progs.consts, X, y, mode, nthreads)


def _ulps(mode, dev_ulps):
    if dev_ulps is None:
        dev_ulps = DEV_ULPS_FP32 if _mode(mode) == FP32 else DEV_ULPS_FP64
    a = np.zeros(64, np.float64)
    for k, v in dev_ulps.items():
        a[k] = v
    return a


def eval_bound(ops, consts, X, mode="fp32", dev_ulps=None):
    """Per-case outputs, per-case error bounds and flags (running error analysis)."""
    ops = np.ascontiguousarray(ops, np.uint8)
    consts = np.ascontiguousarray(consts, np.float32)
    X = np.ascontiguousarray(X, np.float32)
    if X.ndim == 1:
        X = X[None, :]
    d, N = X.shape
    f = np.zeros(N, np.float64)
    dl = np.zeros(N, np.float64)
    u = _ulps(mode, dev_ulps)
    fl = lib().oracle_eval_bound(_p(ops), _p(consts), len(ops), _p(X), N, d, _mode(mode),
                                 _p(u), _p(f), _p(dl))
    return f, dl, int(fl)


def score_bound(progs, X, y, mode="fp32", dev_ulps=None, nthreads: int = 0):
    """(mse, one_minus_r2, flags, mse_bound, one_minus_r2_bound) for a population."""
    ops = np.ascontiguousarray(progs.ops, np.uint8)
    offsets = np.ascontiguousarray(progs.offsets, np.int64)
    lengths = np.ascontiguousarray(progs.lengths, np.int32)
    consts = np.ascontiguousarray(progs.consts, np.float32)
    X = np.ascontiguousarray(X, np.float32)
    if X.ndim == 1:
        X = X[None, :]
    y = np.ascontiguousarray(y, np.float32)
    d, N = X.shape
    P = len(lengths)
    out = [np.zeros(P, np.float64), np.zeros(P, np.float64), np.zeros(P, np.uint32),
           np.zeros(P, np.float64), np.zeros(P, np.float64)]
    u = _ulps(mode, dev_ulps)
    rc = lib().oracle_score_bound(_p(ops), _p(offsets), _p(lengths), _p(consts), P, _p(X),
                                  _p(y), N, d, _mode(mode), _p(u), nthreads, *map(_p, out))
    if rc != 0:
        raise ValueError("oracle_score_bound rejected its arguments")
    return tuple(out)


def eval_cases(ops, consts, X, mode="fp64"):
    """Per-case outputs, per-case invalid markers (uint8) and flags of one program."""
    ops = np.ascontiguousarray(ops, np.uint8)
    consts = np.ascontiguousarray(consts, np.float32)
    X = np.ascontiguousarray(X, np.float32)
    if X.ndim == 1:
        X = X[None, :]
    d, N = X.shape
    f = np.zeros(N, np.float64)
    bad = np.zeros(N, np.uint8)
    fl = lib().oracle_eval_cases(_p(ops), _p(consts), len(ops), _p(X), N, d, _mode(mode),
                                 _p(f), _p(bad))
    return f, bad, int(fl)


def fit_aggregate(f, bad, y, kind, M=10_000, mode="fp64", tax=0.0, length=0, flags=0):
    """(score, asr, r2, taxed, c1, c2, flags) from per-case outputs and invalid markers."""
    f = np.ascontiguousarray(f, np.float64)
    bad = np.ascontiguousarray(bad, np.uint8)
    y = np.ascontiguousarray(y, np.float32)
    out = np.zeros(4, np.float64)
    cnt = np.zeros(2, np.int64)
    fo = ctypes.c_uint32()
    lib().oracle_fit_aggregate(_p(f), _p(bad), _p(y), len(y), flags, kind, M, _mode(mode),
                               tax, length, _p(out), _p(cnt), ctypes.byref(fo))
    return (*out.tolist(), int(cnt[0]), int(cnt[1]), fo.value)


def fit_score(progs, X, y, kind, M=10_000, mode="fp64", tax=0.0, nthreads: int = 0):
    """The paper's fitness of a population: (out [P][4] = score, asr, r2, taxed;
    counts [P][2] = c1, c2; flags [P]). tax < 0 selects the default rate M N / 85."""
    ops = np.ascontiguousarray(progs.ops, np.uint8)
    offsets = np.ascontiguousarray(progs.offsets, np.int64)
    lengths = np.ascontiguousarray(progs.lengths, np.int32)
    consts = np.ascontiguousarray(progs.consts, np.float32)
    X = np.ascontiguousarray(X, np.float32)
    if X.ndim == 1:
        X = X[None, :]
    y = np.ascontiguousarray(y, np.float32)
    d, N = X.shape
    P = len(lengths)
    out = np.zeros((P, 4), np.float64)
    cnt = np.zeros((P, 2), np.int64)
    flags = np.zeros(P, np.uint32)
    rc = lib().oracle_fit_score(_p(ops), _p(offsets), _p(lengths), _p(consts), P, _p(X), _p(y),
                                N, d, _mode(mode), kind, M, tax, nthreads, _p(out), _p(cnt),
                                _p(flags))
    if rc != 0:
        raise ValueError("oracle_fit_score rejected its arguments")
    return out, cnt, flags


TABLE2_CHILDREN = (0.01, 0.03, 0.06, 0.15, 0.25, 0.5, 1.0, 1.5, 2.5, 4.0)


def rank(key, sample, u):
    """Monte-Carlo ranking: (group uint8 [P], children int32 [P]) from keys (higher is
    better), the 100 sampled indices and one uniform number per individual."""
    key = np.ascontiguousarray(key, np.float64)
    sample = np.ascontiguousarray(sample, np.int64)
    u = np.ascontiguousarray(u, np.float32)
    P = len(key)
    group = np.zeros(P, np.uint8)
    children = np.zeros(P, np.int32)
    if lib().oracle_rank(_p(key), P, _p(sample), len(sample), _p(u), _p(group), _p(children)):
        raise ValueError("oracle_rank rejected its arguments")
    return group, children
