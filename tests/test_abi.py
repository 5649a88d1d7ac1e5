"""C-ABI checks that need no GPU: the library loads, exports every function the header
declares, agrees with the generator and the oracle on the wire format, and its host-side
structural check agrees with the oracle's."""
from __future__ import annotations

import ctypes
import re

import numpy as np
import pytest

import oracle
from paper_2607_06731_gb300 import beagle, synth as S
from paper_2607_06731_gb300 import build as B


@pytest.fixture(scope="module", autouse=True)
def built():
    B.build()
    yield


def test_library_exports_every_header_function():
    names = beagle.header_functions()
    assert "beagle_score" in names and "beagle_upload_dataset" in names
    L = ctypes.CDLL(B.LIB)
    for n in names:
        assert hasattr(L, n), n


def test_version_and_error_without_gpu():
    assert beagle.version() == 100
    assert isinstance(beagle.last_error(), str)


def _header_defines():
    out = {}
    for m in re.finditer(r"#define\s+(BEAGLE_\w+)\s+(-?\d+)u?", open(beagle.HEADER).read()):
        out[m.group(1)] = int(m.group(2))
    return out


def test_wire_format_agrees_across_header_generator_and_oracle():
    h = _header_defines()
    names = ["CONST", "ADD", "SUB", "MUL", "PDIV", "SIN", "COS", "EXP", "PLOG", "PSQRT",
             "SQUARE", "DUP", "SWAP", "DEL", "LOAD0", "POW", "SIGN", "CUBE", "CBRT", "TAN",
             "ASIN", "ACOS", "ATAN", "TANH", "COPY0", "PASTE0"]
    for n in names:
        assert h[f"BEAGLE_OP_{n}"] == getattr(S, n), n
    src = open(oracle._SRC).read()
    for n in names:
        m = re.search(rf"\bT_{n}\s*=\s*(\d+)", src)
        assert m and int(m.group(1)) == getattr(S, n), n
    assert h["BEAGLE_MAX_VARS"] == S.MAX_VARS
    assert h["BEAGLE_MAX_REGS"] == S.N_REGS
    m = re.search(r"#define\s+ORACLE_REGS\s+(\d+)", src)
    assert m and int(m.group(1)) == S.N_REGS
    for n, k in (("CORRELATION", oracle.FIT_CORRELATION), ("STD", oracle.FIT_STD),
                 ("STD_SQUARE", oracle.FIT_STD_SQUARE), ("STD_CUBE", oracle.FIT_STD_CUBE),
                 ("STD_HYPER", oracle.FIT_STD_HYPER), ("VALIDATE", oracle.FIT_VALIDATE)):
        assert h[f"BEAGLE_FIT_{n}"] == k == getattr(beagle, f"FIT_{n}"), n
    assert h["BEAGLE_FLAG_PERFECT"] == oracle.F_PERFECT == beagle.FLAG_PERFECT
    assert beagle.FIT_RESULT_DTYPE.itemsize == 56
    assert h["BEAGLE_FLAG_INVALID"] == oracle.F_INVALID
    assert h["BEAGLE_FLAG_DEGENERATE"] == oracle.F_DEGENERATE
    assert h["BEAGLE_FLAG_MALFORMED"] == oracle.F_MALFORMED
    assert beagle.FITNESS_DTYPE.itemsize == 24


def test_host_validation_agrees_with_oracle():
    rng = np.random.default_rng(5)
    ok = S.gen_programs(rng, 300, 1, 60, 3)
    assert beagle.validate_programs(ok.ops, ok.offsets, ok.lengths, 3) == -1
    alphabet = np.array([S.CONST, S.ADD, S.SUB, S.SIN, S.DUP, S.SWAP, S.DEL, S.LOAD0,
                         S.LOAD0 + 2, S.LOAD0 + 3, S.POW, S.TANH, S.COPY0, S.COPY0 + 1,
                         S.PASTE0, S.PASTE0 + 1, 23, 99], np.uint8)
    for _ in range(3000):
        L = int(rng.integers(1, 9))
        ops = rng.choice(alphabet, L).astype(np.uint8)
        want = oracle.check_program(ops, 3, 16)
        got = beagle.validate_programs(ops, np.zeros(1, np.int64), np.array([L], np.int32), 3)
        assert (got == -1) == (want == 0), (ops, want, got)
    # depth limit and length limit
    deep = np.array([S.CONST] * 17 + [S.ADD] * 16, np.uint8)
    assert beagle.validate_programs(deep, [0], [len(deep)], 1, max_depth=16) == 0
    assert beagle.validate_programs(deep, [0], [len(deep)], 1) == -1     # default: 32
    deeper = np.array([S.CONST] * 33 + [S.ADD] * 32, np.uint8)
    assert beagle.validate_programs(deeper, [0], [len(deeper)], 1) == 0
    long = np.array([S.CONST] + [S.SIN] * 256, np.uint8)
    assert beagle.validate_programs(long, [0], [257], 1, max_depth=32) == 0


def test_operator_whitelist():
    """GetAllowedOperations' analogue: a program using an operator outside the list fails."""
    progs = S.from_token_lists([[(S.LOAD0, 0.0), (S.SIN, 0.0)],
                                [(S.LOAD0, 0.0), (S.COPY0, 0.0), (S.PASTE0, 0.0), (S.MUL, 0.0)],
                                [(S.CONST, 1.0), (S.LOAD0 + 1, 0.0), (S.POW, 0.0)]])
    args = (progs.ops, progs.offsets, progs.lengths, 2)
    assert beagle.validate_programs(*args) == -1
    assert beagle.validate_programs(*args, allowed=[S.LOAD0, S.CONST, S.SIN, S.MUL, S.POW,
                                                    S.COPY0]) == -1
    assert beagle.validate_programs(*args, allowed=[S.LOAD0, S.SIN, S.MUL, S.COPY0]) == 2
    assert beagle.validate_programs(*args, allowed=[S.LOAD0, S.SIN, S.CONST, S.POW]) == 1
    unary, binary = S.allowed_operations(exclude=(S.SIN, S.COS))
    assert S.SIN not in unary and S.COS not in unary and S.TANH in unary and S.POW in binary
    gen = S.gen_programs(np.random.default_rng(1), 200, 4, 30, 2, unary=unary, binary=binary)
    assert not np.isin(gen.ops, [S.SIN, S.COS]).any()
    assert beagle.validate_programs(gen.ops, gen.offsets, gen.lengths, 2,
                                    allowed=[S.CONST, S.LOAD0, *unary, *binary]) == -1


def test_score_rejects_unknown_dataset_without_touching_a_gpu():
    rc = beagle.lib().beagle_score(None, None, None, None, 0, 12345, None, 0, None)
    assert rc == -3
    assert "unknown dataset" in beagle.last_error()
    rc = beagle.lib().beagle_score(None, None, None, None, 0, 12345, None, 7, None)
    assert rc == -1


def test_batch_api_argument_checks_without_a_gpu():
    assert beagle.lib().beagle_score_batch(None, -1, 0, None) == -1
    assert beagle.lib().beagle_score_batch(None, 0, 0, None) == 0
    jobs = beagle.Job * 1
    arr = jobs()
    arr[0].dataset_id = 424242
    arr[0].P = 5
    assert beagle.lib().beagle_score_batch(arr, 1, 0, None) == -3
    assert beagle.lib().beagle_batch_plan_launch(None, None) == -1
    assert beagle.lib().beagle_batch_plan_destroy(None) == 0
    cfg = beagle.LaunchConfig(3, 0, 0, 0, 0, 0)
    assert beagle.lib().beagle_set_launch_config(ctypes.byref(cfg)) == -1


def test_serve_api_argument_checks_without_a_gpu():
    L = beagle.lib()
    assert L.beagle_serve_create(None, None) == -1
    cfg = beagle.ServeConfig(1 << 20, 2, 8, 7, 0)
    h = ctypes.c_void_p()
    assert L.beagle_serve_create(ctypes.byref(cfg), ctypes.byref(h)) == -1
    assert "precision" in beagle.last_error()
    cfg = beagle.ServeConfig(1 << 20, 9, 8, 0, 0)
    assert L.beagle_serve_create(ctypes.byref(cfg), ctypes.byref(h)) == -8
    assert L.beagle_serve_submit(None, None, None) == -1
    assert L.beagle_serve_stats(None, None) == -1
    assert L.beagle_serve_wait(None, 1, None, 0) == -1
    assert L.beagle_serve_destroy(None) == 0
    assert ctypes.sizeof(beagle.ServeConfig) == 24
    assert ctypes.sizeof(beagle.Request) == 56
    assert ctypes.sizeof(beagle.ServeStats) == 10 * 8 + 4 * 8


def test_early_exit_and_case_counter_settings_without_a_gpu():
    """beagle_set_invalid_early_exit and beagle_count_cases are host settings: they take no
    device work; a counter array needs a positive population size."""
    L = beagle.lib()
    assert L.beagle_set_invalid_early_exit(0) == 0
    assert L.beagle_set_invalid_early_exit(1) == 0
    assert L.beagle_count_cases(1, 0) == -1          # BEAGLE_ERR_ARG
    assert L.beagle_count_cases(1, -5) == -1
    assert L.beagle_count_cases(None, 0) == 0        # off
