"""Host logic of bench.py that needs no GPU: the parity gates' program selection and the
count of the operators the packing kernel folds."""
from __future__ import annotations

import numpy as np

import bench
from paper_2607_06731_gb300 import synth as S


def _oracle(n):
    z = {k: np.full(n, 1.0) for k in ("fp32_mse", "fp32_omr2", "fp64_mse", "fp64_omr2")}
    for k in ("fp32_bm", "fp32_br", "fp64_bm", "fp64_br"):
        z[k] = np.zeros(n)
    z["fp32_flags"] = np.zeros(n, np.uint32)
    z["fp64_flags"] = np.zeros(n, np.uint32)
    return z


def test_parity_gates_strict_set():
    """Gate A and B count only programs whose FP32-ops bound is tight; gate C those whose FP64
    bound is; a loose program outside the gates does not fail them."""
    o = _oracle(4)
    o["fp32_bm"][1] = 1e-3          # fp32-sensitive: out of gates A/B
    o["fp64_bm"][2] = 1e-10         # out of gate C (fp64 bound above 1e-13)
    g32 = (np.array([1.0, 1.5, 1.0, 1.0]), np.ones(4), np.zeros(4, np.uint32))
    g64 = (np.array([1.0, 1.0, 1.0 + 1e-11, 1.0]), np.ones(4), np.zeros(4, np.uint32))
    out = bench.parity_gates(g32, g64, o)
    assert out["gate_A"]["of"] == 3 and out["gate_A"]["pass"] == 3
    assert out["gate_C"]["of"] == 3 and out["gate_C"]["pass"] == 3
    assert out["all_pass"]
    g32[0][0] = 1.001               # a strict program off by 1e-3: gate A fails
    out = bench.parity_gates(g32, g64, o)
    assert out["gate_A"]["pass"] == 2 and out["gate_A"]["failing_sample_positions"] == [0]
    assert not out["all_pass"]


def test_folded_op_counts_match_a_sequential_fold():
    """The vectorised count of folded operators equals a plain stack walk over every program
    (an operator is folded when all its operands are constants; DUP, SWAP, DEL of constants
    too; programs with COPY/PASTE are left alone)."""
    rng = np.random.default_rng(5)
    progs = S.gen_programs(rng, 400, 3, 60, 3, unary=S.ALL_UNARY, binary=S.ALL_BINARY)
    progs = S.with_registers(progs, 3, 0.2, 2)   # register programs are not folded
    got = bench.folded_op_counts(progs)
    want = np.zeros(256, np.int64)
    un = set(range(S.SIN, S.SQUARE + 1)) | set(range(S.POW + 1, S.TANH + 1))
    bn = {S.ADD, S.SUB, S.MUL, S.PDIV, S.POW}
    for p in range(progs.P):
        ops = list(progs.program(p)[0])
        if any(S.COPY0 <= op < S.PASTE0 + 16 for op in ops):
            continue
        st = []
        for op in ops:
            if op == S.CONST:
                st.append(True)
            elif S.LOAD0 <= op < S.LOAD0 + 16:
                st.append(False)
            elif op in un:
                if st[-1]:
                    want[op] += 1
            elif op in bn:
                b, a = st.pop(), st.pop()
                st.append(a and b)
                if a and b:
                    want[op] += 1
    assert np.array_equal(got, want)
    assert want.sum() > 0


def test_case_weights_scale_the_executed_work():
    """The roofline's units and the executed node count follow each program's share of the
    cases it ran (beagle_count_cases): every case gives the unweighted counts; a program that
    ran half its cases counts half; one that ran none, nothing."""
    rng = np.random.default_rng(8)
    progs = S.gen_programs(rng, 300, 3, 40, 3)
    N = 1 << 15                                    # P N below 2^24: no folding
    ones = np.ones(progs.P)
    assert np.array_equal(bench.op_counts(progs, ones), bench.op_counts(progs))
    assert np.allclose(bench.folded_op_counts(progs, ones), bench.folded_op_counts(progs))
    full = bench.algorithmic_units([(progs, N)], folded=True)
    same = bench.algorithmic_units([(progs, N, ones)], folded=True)
    half = bench.algorithmic_units([(progs, N, 0.5 * ones)], folded=True)
    for k in full:
        assert np.isclose(same[k], full[k]) and np.isclose(half[k], 0.5 * full[k])
    w = np.zeros(progs.P)
    w[0] = 1.0
    one = bench.algorithmic_units([(progs, N, w)], folded=False)
    alone = bench.algorithmic_units([(progs.subset(np.array([0])), N)], folded=False)
    for k in one:
        assert np.isclose(one[k], alone[k])
    cases = np.full(progs.P, N, np.int64)
    cases[: progs.P // 2] = N // 4
    info = bench.work_info(progs, N, cases, ms=2.0)
    L = progs.lengths.astype(np.float64)
    want = (L[: progs.P // 2].sum() * (N // 4) + L[progs.P // 2:].sum() * N)
    assert np.isclose(info["executed_node_evals_per_step"], want)
    assert np.isclose(info["executed_case_fraction"], cases.sum() / (progs.P * N))
    assert np.isclose(info["executed_gpops"], want / 2e-3 / 1e9)
    assert bench.work_info(progs, N)["executed_node_evals_per_step"] == L.sum() * N
