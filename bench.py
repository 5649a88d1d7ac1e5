#!/usr/bin/env python3
"""Population fitness scoring benchmark: GPoPs (program-node evaluations per second).

One step = one beagle_score call over a whole population: every program interpreted on
every fitness case and reduced to its MSE and 1 - r^2 (Beagle tutorial, "Dividing Tasks
Between CPU and GPU": one aggregated fitness per individual). The default run is the
precision workload: P = 50,000 random postfix programs (length U{16..64}, d = 10 inputs) on
N = 1,000,000 fitness cases, X ~ N(0, 1), y = a random 30-node expression scaled to RMS 1e3
plus N(0, 1) noise, on the FP32-compensated path, with the plain FP64 path beside it and the
oracle's verdict on a seeded 10,000-program sample at the full case count. The same line
carries compact sub-lines for the small oracle-sized case, the 100,000-program population and
the 64 ragged populations in one graph-captured batch. Inputs are resident in HBM before
timing; L2 is flushed (a 256 MiB write) before every timed step, outside the timed events.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload headline|c1|c2|c3|c4|c5]

Under torchrun each rank scores its own population (seed + rank) on its own GPU with no
collective on the data path (weak scaling); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import multiprocessing as mp
import os
import shutil
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "GPoPs (node-evals/s) FP32-compensated vs plain FP64 at ≤1e-5 rel err; p50/p99"
# Kernels one scoring call launches: on launches of at least 2^24 program-cases the length sort
# (two kernels) and packing (each program translated into handlers once, constants folded),
# then on every launch the persistent scoring kernel's fast pass and deep pass (programs deeper
# than 16 values; it exits at once when there are none) and the fp64 finalize.
PACKED_LAUNCH_CASES = 1 << 24


def launches_per_call(P: int, N: int) -> int:
    return 6 if P * N >= PACKED_LAUNCH_CASES else 3
C1_DESC = ("c1-small-1024: P=1024 programs, length U{8..32}, d=2, N=1024 cases, X~U[-3,3], "
           "y = x0 sin(x1) + x0^2/2; MSE")
C2_DESC = ("c2-population-100k: P=100000 programs, length U{16..128}, d=5, N=1024 cases, "
           "X~U[-3,3], y=20-node expression + N(0,0.01) noise; MSE and 1-R^2")
C3_DESC = ("c3-precision-1m: P=50000 programs, length U{16..64}, d=10, N=1000000 cases, "
           "X~N(0,1), y=30-node expression at RMS 1e3 + N(0,1) noise; FP32-compensated vs "
           "plain FP64, error against the FP64 oracle on a 10k-program sample")
C4_DESC = ("c4-ragged-64: 64 populations, P log-U[1e3,2e5], L U{4..256}, N log-U[256,1e5], "
           "d U{1..10}, one dataset each; one graph-captured batch per step")


def parse():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=["headline", "c1", "c2", "c3", "c4", "c5", "handlers"],
                    default="headline",
                    help="headline (default): the precision workload with oracle gates and "
                         "compact c1/c2/c4 sub-lines; c1..c5: one workload on its own line; "
                         "handlers: one scoring launch per interpreter handler (programs "
                         "repeating it) for instruction counts under ncu")
    ap.add_argument("--fp64-steps", type=int, default=1)
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--parity-sample", type=int, default=10_000,
                    help="programs of the timed launch checked against the oracle at the full "
                         "case count (0: skip)")
    ap.add_argument("--cpu-seconds", type=float, default=10.0,
                    help="target wall time of the CPU oracle sample")
    ap.add_argument("--P", type=int, default=0, help="override the population size")
    ap.add_argument("--requests", type=int, default=200, help="c5: requests per load level")
    ap.add_argument("--autotune", action="store_true",
                    help="let beagle_autotune pick the launch shape before timing")
    ap.add_argument("--no-sub", action="store_true", help="headline without the sub-lines")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class Clocks:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(sm)}


# ----------------------------------------------------------------------------- roofline
# Algorithmic operations per node evaluation (the method's own arithmetic; leaves and stack
# moves cost nothing), by opcode: (FP32 pipe, MUFU/XU pipe, ALU pipe) lane operations. Every
# operator also pays one validity compare on the ALU pipe.
#   add/sub/mul/square  1 FP32                    + 1 ALU
#   protected divide    3 FP32 + 1 MUFU (rcp)     + 2 ALU (threshold select, validity)
#   sin, cos            4 FP32 + 1 MUFU           + 1 ALU
#   exp                 2 FP32 + 1 MUFU (ex2)     + 1 ALU
#   protected log       1 FP32 + 1 MUFU (lg2)     + 2 ALU (threshold select, validity)
#   protected sqrt      2 FP32 + 1 MUFU (rsq)     + 1 ALU
ALGO_UNITS = {1: (1, 0, 1), 2: (1, 0, 1), 3: (1, 0, 1), 10: (1, 0, 1),
              4: (3, 1, 2), 5: (4, 1, 1), 6: (4, 1, 1), 7: (2, 1, 1), 8: (1, 1, 2),
              9: (2, 1, 1)}
# Lanes per SM per clock of each pipe on GB300 (ncu .peak_sustained: FMA 4, ALU 2, XU 1 warp
# instructions per SM per cycle) and the issue limit (4 warp instructions per SM per cycle).
LANES_PER_SM_CLK = {"fp32": 128, "mufu": 32, "alu": 64, "issue": 128}


def folded_op_counts(progs, w=None):
    """Per opcode, the operators the packing kernel folds (constant subexpressions, evaluated
    once per call instead of on every case): the constness of every stack value followed
    through all programs at once, token position by token position. As on the device, only
    programs of leaves, unary and binary operators are folded. w: optional per-program
    weights (each program's folded operators count w[p] times)."""
    from paper_2607_06731_gb300 import synth as S
    P = progs.P
    out = np.zeros(256, np.float64 if w is not None else np.int64)
    if P == 0:
        return out
    L = progs.lengths.astype(np.int64)
    offs = progs.offsets.astype(np.int64)
    cst = np.zeros((P, 36), bool)
    sp = np.zeros(P, np.int64)
    other = np.zeros(P, bool)   # DUP, SWAP, DEL, COPY/PASTE or unknown: not folded
    per = []
    un = np.zeros(256, bool)
    for op in list(range(S.SIN, S.SQUARE + 1)) + list(range(S.POW + 1, S.TANH + 1)):
        un[op] = True
    bn = np.zeros(256, bool)
    bn[[S.ADD, S.SUB, S.MUL, S.PDIV, S.POW]] = True
    for t in range(int(L.max())):
        act = np.nonzero(L > t)[0]
        op = progs.ops[offs[act] + t].astype(np.int64)
        s_ = sp[act]
        isconst = op == S.CONST
        isvar = (op >= S.LOAD0) & (op < S.LOAD0 + 16)
        u, b = un[op], bn[op]
        other[act[~(isconst | isvar | u | b)]] = True
        lf = isconst | isvar
        cst[act[lf], np.minimum(s_[lf], 35)] = isconst[lf]
        fu = u & cst[act, np.maximum(s_ - 1, 0)]
        both = cst[act, np.maximum(s_ - 1, 0)] & cst[act, np.maximum(s_ - 2, 0)]
        fb = b & both
        cst[act[b], np.maximum(s_[b] - 2, 0)] = both[b]
        sp[act] += lf.astype(np.int64) - b
        f = fu | fb
        per.append((act[f], op[f]))
    for idx, op in per:
        keep = ~other[idx]
        np.add.at(out, op[keep], 1 if w is None else w[idx[keep]])
    return out


def op_counts(progs, w=None):
    """Per opcode, the operators of the programs (each program's counted w[p] times)."""
    if w is None:
        return np.bincount(progs.ops, minlength=256).astype(np.float64)
    tw = np.repeat(np.asarray(w, np.float64), progs.lengths.astype(np.int64))
    return np.bincount(progs.ops, weights=tw, minlength=256)


def removed_tokens(folded):
    """Tokens folding removes: one per folded unary operator (CONST U -> CONST), two per
    folded binary one (CONST CONST B -> CONST)."""
    from paper_2607_06731_gb300 import synth as S
    bins = [S.ADD, S.SUB, S.MUL, S.PDIV, S.POW]
    nb = int(folded[bins].sum())
    return int(folded.sum()) + nb


def launch_folds(P: int, N: int) -> bool:
    """Whether a launch of this size runs the packing kernel (and so folds constants)."""
    return P * N >= PACKED_LAUNCH_CASES


def case_weights(cases_run, N):
    """Per program, the fraction of the N fitness cases the scoring call evaluated
    (beagle_count_cases), or None (every case)."""
    return None if cases_run is None else np.asarray(cases_run, np.float64) / float(N)


def work_info(progs, N, cases_run=None, ms=None):
    """The config entries on the work a step does: node evaluations of the original programs
    (the metric's count), and of what the interpreter ran: constant subexpressions folded
    once per call, and the cases each program ran (an invalid program stops at the first
    case tile pass that meets an invalid value; its later tiles are not run)."""
    tok = float(progs.lengths.sum(dtype=np.int64))
    ev = tok * N
    w = case_weights(cases_run, N)
    folds = launch_folds(progs.P, N)
    ran = float(np.dot(progs.lengths.astype(np.float64), w)) if w is not None else tok
    rm = removed_tokens(folded_op_counts(progs, w)) if folds else 0.0
    out = {"constant_folding": ("on: constant subexpressions evaluated once per call by the "
                                "packing kernel, same bits" if folds else
                                "off (launch below 2^24 program-cases)"),
           "invalid_early_exit": ("on: a program stops at the first case pass with an invalid "
                                  "value, later tiles of a program found invalid are skipped; "
                                  "same bits (the validity rule makes it invalid whatever its "
                                  "other cases give)" if w is not None else "not measured"),
           "value_counts": "node evaluations of the original programs on every case",
           "executed_node_evals_per_step": (ran - float(rm)) * N}
    if folds:
        out["folded_token_fraction"] = removed_tokens(folded_op_counts(progs)) / max(1.0, tok)
    if w is not None:
        out["executed_case_fraction"] = float(np.sum(cases_run)) / max(1.0, float(progs.P) * N)
        if ms:
            out["executed_gpops"] = out["executed_node_evals_per_step"] / (ms / 1e3) / 1e9
    return out


def algorithmic_units(progs_list, folded=True):
    """Lane operations of each pipe over populations [(programs, N[, w])], of the operators
    the interpreter runs: the folded constant subexpressions left out when folded, and each
    program's operators on the fraction w[p] of the cases it ran (all when w is absent)."""
    tot = {"fp32": 0.0, "mufu": 0.0, "alu": 0.0}
    for item in progs_list:
        progs, N = item[0], item[1]
        w = item[2] if len(item) > 2 else None
        counts = op_counts(progs, w)
        if folded:
            counts -= folded_op_counts(progs, w)
        for op, (f, m, a) in ALGO_UNITS.items():
            tot["fp32"] += counts[op] * N * f
            tot["mufu"] += counts[op] * N * m
            tot["alu"] += counts[op] * N * a
    tot["issue"] = tot["fp32"] + tot["mufu"] + tot["alu"]
    return tot


def roofline_time(progs_list, sm_mhz: float, sms: int, folded=True):
    """Roofline time of the populations' algorithmic work: the slowest of the FP32, MUFU and
    ALU pipes and of instruction issue, at the measured SM clock."""
    units = algorithmic_units(progs_list, folded)
    f = sm_mhz * 1e6
    t = {k: units[k] / (LANES_PER_SM_CLK[k] * sms * f) for k in units}
    bind = max(t, key=t.get)
    return {"seconds": t[bind], "binding": bind, "per_pipe_ms": {k: v * 1e3 for k, v in t.items()},
            "lane_ops_per_node_eval": units["issue"] / max(1.0, sum(
                float(it[0].lengths.sum(dtype=np.int64)) * it[1] for it in progs_list))}


def roofline_line(node_evals, kernel_s, progs_list, sm_mhz, sms, peak_straight=None,
                  folded=True):
    rt = roofline_time(progs_list, sm_mhz, sms, folded)
    peak = node_evals / rt["seconds"] / 1e9
    achieved = node_evals / kernel_s / 1e9 if kernel_s else None
    out = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "GPoPs",
           "frac": achieved / peak if achieved else None, "traffic": None,
           "peak_basis": (f"algorithmic lane operations per node evaluation (FP32/MUFU/ALU "
                          f"units per operator, leaves free) of the operators and cases the "
                          f"kernels ran, at {LANES_PER_SM_CLK} lanes per SM per clock, {sms} "
                          f"SMs, {sm_mhz:.0f} MHz measured; binding: {rt['binding']}"),
           "per_pipe_ms": rt["per_pipe_ms"],
           "lane_ops_per_node_eval": rt["lane_ops_per_node_eval"],
           "kernel_ms": kernel_s * 1e3 if kernel_s else None}
    if peak_straight:
        out["peak_straight_line_ops"] = peak_straight
        out["frac_straight_line_ops"] = achieved / peak_straight if achieved else None
    return out


def straight_line_peak(progs, N, rates, folded=True, w=None):
    """Seconds straight-line compiled code would need for this op mix (the operators and cases
    the interpreter runs: folded constant subexpressions left out when folded, each program on
    the fraction w[p] of the cases it ran), every operator at its measured throughput
    (beagle_measure_op_rates), leaves free."""
    counts = op_counts(progs, w)
    if folded:
        counts -= folded_op_counts(progs, w)
    return sum(counts[op] * N / r for op, r in rates.items())


# ----------------------------------------------------------------------------- oracle legs
# The oracle (test infrastructure) runs only here, outside every timed region: the CPU
# baseline, the reference arm, and the parity gates on a sample of the timed launch's output.
def _oracle_worker(inp: str, outp: str):
    """Spawned process: FP32-ops and FP64 oracle results of a program sample, each with its
    running error bound (the bound of a device computing in that precision with its
    transcendentals' ulps)."""
    sys.path.insert(0, ROOT)
    import oracle
    from paper_2607_06731_gb300 import synth
    oracle.build()
    z = np.load(inp)
    res = {}
    t0 = time.perf_counter()
    progs = synth.Programs(z["ops"], z["offsets"], z["lengths"], z["consts"])
    m, r, f, bm, br = oracle.score_bound(progs, z["X"], z["y"], "fp32")
    res["fp32_mse"], res["fp32_omr2"], res["fp32_flags"] = m, r, f
    res["fp32_bm"], res["fp32_br"] = bm, br
    m, r, f, bm, br = oracle.score_bound(progs, z["X"], z["y"], "fp64")
    res["fp64_mse"], res["fp64_omr2"], res["fp64_flags"] = m, r, f
    res["fp64_bm"], res["fp64_br"] = bm, br
    res["seconds"] = np.array(time.perf_counter() - t0)
    res["threads"] = np.array(oracle.threads())
    np.savez(outp, **res)


class OracleSample:
    """The oracle on a seeded sample of a population, in a spawned process (started before
    any GPU work, so that it overlaps the timed runs)."""

    def __init__(self, pr, n: int, seed: int = 11):
        self.idx = np.sort(np.random.default_rng(seed).choice(pr.programs.P,
                                                              min(n, pr.programs.P),
                                                              replace=False))
        sub = pr.programs.subset(self.idx)
        self.dir = tempfile.mkdtemp(prefix="beagle_parity_")
        inp = os.path.join(self.dir, "in.npz")
        np.savez(inp, ops=sub.ops, offsets=sub.offsets, lengths=sub.lengths, consts=sub.consts,
                 X=pr.X, y=pr.y)
        self.out = os.path.join(self.dir, "out.npz")
        self.proc = mp.get_context("spawn").Process(target=_oracle_worker,
                                                    args=(inp, self.out))
        self.t0 = time.perf_counter()
        self.proc.start()

    def result(self):
        self.proc.join()
        wall = time.perf_counter() - self.t0
        if self.proc.exitcode != 0:
            shutil.rmtree(self.dir, ignore_errors=True)
            raise RuntimeError(f"oracle sample process failed ({self.proc.exitcode})")
        z = dict(np.load(self.out))
        shutil.rmtree(self.dir, ignore_errors=True)
        z["wall"] = wall
        return z


def oracle_inline(progs, X, y):
    import oracle
    oracle.build()
    res = {}
    m, r, f, bm, br = oracle.score_bound(progs, X, y, "fp32")
    res["fp32_mse"], res["fp32_omr2"], res["fp32_flags"] = m, r, f
    res["fp32_bm"], res["fp32_br"] = bm, br
    m, r, f, bm, br = oracle.score_bound(progs, X, y, "fp64")
    res["fp64_mse"], res["fp64_omr2"], res["fp64_flags"] = m, r, f
    res["fp64_bm"], res["fp64_br"] = bm, br
    return res


def _close(a, b, rel, abs_):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    inf = np.isinf(a) & np.isinf(b) & (np.sign(a) == np.sign(b))
    with np.errstate(invalid="ignore"):
        return (np.abs(a - b) <= np.maximum(rel * np.abs(b), abs_)) | inf


def _max_rel(a, b):
    if len(a) == 0:
        return None
    with np.errstate(invalid="ignore", divide="ignore"):
        r = np.abs(a - b) / np.maximum(np.abs(b), 1e-300)
    return float(np.max(r))


def parity_gates(g32, g64, o):
    """Gates A, B, C against the oracle. NEAR: the oracle saw a value within 1e-5 of a
    threshold (1e30, 1e-3), where fp32 and fp64 may decide differently; AMBIGUOUS: a decision
    lies inside the FP64 oracle's running error bound. The strict (well-conditioned) set for
    the FP32 path, as in the tests: valid, neither, the FP32-ops oracle's error bound within
    1e-6 (a device whose fp32 transcendentals are within their ulp limits lands within 1e-6 of
    the FP32-ops oracle), the FP32-ops and FP64 oracle results agree within 1e-6, and the FP64
    error bound is within 1e-9 (no chaotic sensitivity that the fp32 comparison could miss).
      flags   GPU flags equal the oracle's on every program neither NEAR nor AMBIGUOUS
      gate A  GPU FP32c vs FP32-ops oracle, |g - o| <= max(1e-5 |o|, 1e-7), strict set
      gate B  GPU FP32c vs FP64 oracle, same tolerance, strict set
      gate C  GPU FP64 vs FP64 oracle, |g - o| <= max(1e-12 |o|, 1e-13), on the valid,
              decided programs whose FP64 bound is within 1e-13 (as in the tests)"""
    NEAR, AMBIG, BITS = 256, 512, 7
    f32, f64 = o["fp32_flags"].astype(np.int64), o["fp64_flags"].astype(np.int64)
    near = ((f32 | f64) & NEAR) != 0
    amb = (f64 & AMBIG) != 0
    valid = ((f32 & 5) == 0) & ((f64 & 5) == 0)
    m64, r64, bm, br = o["fp64_mse"], o["fp64_omr2"], o["fp64_bm"], o["fp64_br"]
    agree = (_close(o["fp32_mse"], m64, 1e-6, 1e-9) & _close(o["fp32_omr2"], r64, 1e-6, 1e-9) &
             ((f32 & BITS) == (f64 & BITS)))
    with np.errstate(invalid="ignore"):
        tight9 = (bm <= 1e-9 * np.abs(m64) + 1e-12) & (br <= 1e-9 * np.abs(r64) + 1e-12)
        tight13 = (bm <= 1e-13 * np.abs(m64) + 1e-15) & (br <= 1e-13 * np.abs(r64) + 1e-15)
        m32, r32 = o["fp32_mse"], o["fp32_omr2"]
        tight32 = ((o["fp32_bm"] <= 1e-6 * np.abs(m32) + 1e-9) &
                   (o["fp32_br"] <= 1e-6 * np.abs(r32) + 1e-9))
    strict = valid & ~near & ~amb & agree & tight9 & tight32
    strict_c = valid & ~near & ~amb & tight13   # the FP64 path: its own bound decides
    decided = ~near & ~amb
    out = {"programs": int(len(f32)), "valid": int(valid.sum()), "near_threshold": int(near.sum()),
           "ambiguous": int(amb.sum()), "strict": int(strict.sum()),
           "strict_frac": float(strict.mean()) if len(f32) else None,
           "strict_fp64": int(strict_c.sum())}
    fl32 = int(np.sum(decided & ((g32[2].astype(np.int64) & BITS) != (f32 & BITS))))
    out["flags_mismatch_fp32"] = fl32
    ok_all = fl32 == 0
    for name, g, mse, omr, tol, sel in (
            ("A", g32, "fp32_mse", "fp32_omr2", (1e-5, 1e-7), strict),
            ("B", g32, "fp64_mse", "fp64_omr2", (1e-5, 1e-7), strict),
            ("C", g64, "fp64_mse", "fp64_omr2", (1e-12, 1e-13), strict_c)):
        if g is None:
            continue
        ok = _close(g[0], o[mse], *tol) & _close(g[1], o[omr], *tol)
        npass = int(np.sum(ok & sel))
        fails = np.nonzero(sel & ~ok)[0]
        out[f"gate_{name}"] = {"pass": npass, "of": int(sel.sum()),
                               "tol_rel": tol[0], "tol_abs": tol[1],
                               "max_rel_mse": _max_rel(g[0][sel], o[mse][sel]),
                               "max_rel_one_minus_r2": _max_rel(g[1][sel], o[omr][sel]),
                               "failing_sample_positions": fails[:16].tolist()}
        ok_all &= npass == int(sel.sum())
    if g64 is not None:
        fl64 = int(np.sum(decided & ((g64[2].astype(np.int64) & BITS) != (f64 & BITS))))
        out["flags_mismatch_fp64"] = fl64
        ok_all &= fl64 == 0
    # outside the strict set: how far FP32c lands from the FP64 oracle (conditioning of the
    # programs themselves, not the aggregation)
    rest = valid & decided & ~strict & ((g32[2] & 5) == 0)
    if rest.any():
        ok = _close(g32[0], m64, 1e-5, 1e-7) & _close(g32[1], r64, 1e-5, 1e-7)
        out["outside_strict_within_1e-5_of_fp64"] = float(np.mean(ok[rest]))
    out["all_pass"] = bool(ok_all)
    return out


def cpu_baseline(pr, seconds: float, threads: int = 0):
    """Time the oracle (FP64, as it stands) on a seeded sample of the population."""
    import oracle
    oracle.build()
    rng = np.random.default_rng(1234)
    mean_len = float(pr.programs.lengths.mean())
    n = int(min(pr.programs.P, max(2, min(200, 2e8 / (mean_len * pr.N)))))
    # sample sizes scaled from the previous run's time until a run takes at least half the
    # target (the first, small run also pays the thread pool's start)
    n2 = n
    for _ in range(4):
        idx = rng.choice(pr.programs.P, n2, replace=False)
        sub = pr.programs.subset(idx)
        t0 = time.perf_counter()
        oracle.score_programs(sub, pr.X, pr.y, "fp64", nthreads=threads)
        dt = max(time.perf_counter() - t0, 1e-6)
        if dt >= 0.5 * seconds or n2 >= pr.programs.P:
            break
        n2 = int(min(pr.programs.P, max(n2 + 1, n2 * seconds / dt)))
    evals = int(sub.lengths.sum()) * pr.N
    out = {"value": evals / dt / 1e9, "unit": "GPoPs", "cores": oracle.threads(),
           "kind": "oracle",
           "sample": f"{n2} of {pr.programs.P} programs (seeded) x all {pr.N} cases, FP64 "
                     f"oracle, {dt:.1f} s wall"}
    if threads == 0:   # the same oracle on one core, on a sample of about a fifth of the time
        n1 = max(2, n2 // (5 * max(1, oracle.threads())))
        sub1 = pr.programs.subset(idx[:n1])
        t0 = time.perf_counter()
        oracle.score_programs(sub1, pr.X, pr.y, "fp64", nthreads=1)
        dt1 = time.perf_counter() - t0
        out["single_core"] = {"value": int(sub1.lengths.sum()) * pr.N / dt1 / 1e9,
                              "unit": "GPoPs", "sample": f"{n1} programs, {dt1:.1f} s wall"}
    return out


def run_reference(args, rank, world):
    """The oracle timed as the reference arm on the headline workload: each step scores a
    bounded seeded sample of the precision population at the full case count."""
    if rank != 0:
        return 0
    from paper_2607_06731_gb300 import synth
    import oracle
    oracle.build()
    pr = synth.make_c3(P=args.P or 50_000)
    rng = np.random.default_rng(99)
    n = 16
    sub = pr.programs.subset(rng.choice(pr.programs.P, n, replace=False))
    t0 = time.perf_counter()
    oracle.score_programs(sub, pr.X, pr.y, "fp64")
    dt = max(time.perf_counter() - t0, 1e-6)
    per_step = max(1.0, min(8.0, 150.0 / max(1, args.steps + args.warmup)))
    n = int(min(pr.programs.P, max(n, n * per_step / dt)))
    sub = pr.programs.subset(rng.choice(pr.programs.P, n, replace=False))
    evals = int(sub.lengths.sum()) * pr.N
    for _ in range(args.warmup):
        oracle.score_programs(sub, pr.X, pr.y, "fp64")
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.score_programs(sub, pr.X, pr.y, "fp64")
        times.append(time.perf_counter() - t0)
    tot = sum(times)
    value = evals * args.steps / tot / 1e9
    sample = f"{n} of {pr.programs.P} programs (seeded) x all {pr.N} cases per step, FP64"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "GPoPs",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": tot / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": C3_DESC, "P": pr.programs.P, "N": pr.N, "d": pr.d,
                       "sample_programs": n},
            "cpu_baseline": {"value": value, "unit": "GPoPs", "cores": oracle.threads(),
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "GPoPs", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------------------- GPU legs
def timed_steps(step, steps, warmup, stream, flush, barrier=None):
    """W untimed warm-up steps, then K steps each between CUDA events on the launching
    stream, L2 flushed before every step outside the events. Returns per-step ms."""
    import torch
    for _ in range(warmup):
        flush.zero_()
        step()
    torch.cuda.synchronize()
    if barrier:
        barrier()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(steps)]
    for a, b in evs:
        flush.zero_()
        a.record(stream)
        step()
        b.record(stream)
    torch.cuda.synchronize()
    if barrier:
        barrier()
    return [a.elapsed_time(b) for a, b in evs]


def _pctl(v, q):
    v = sorted(v)
    return v[min(len(v) - 1, int(round(q * (len(v) - 1))))] if v else None


def e2e_host(beagle, progs, ds, stream, steps):
    """GPoPs end to end through beagle_score_host: programs from pinned host memory to the
    device and the fitness records back, inside the timed region (the dataset is resident)."""
    import torch
    from paper_2607_06731_gb300 import synth
    pinned = [torch.from_numpy(np.ascontiguousarray(a)).pin_memory() for a in
              (progs.ops, progs.offsets, progs.lengths, progs.consts)]
    hp = synth.Programs(*(t.numpy() for t in pinned))
    hout = torch.empty(progs.P * 3, dtype=torch.float64).pin_memory()
    hout_np = hout.numpy().view(beagle.FITNESS_DTYPE)
    beagle.score_host(hp, ds, out=hout_np, stream=stream)
    ts = []
    for _ in range(steps):
        t0 = time.perf_counter()
        beagle.score_host(hp, ds, out=hout_np, stream=stream)
        ts.append(time.perf_counter() - t0)
    h2d = hp.ops.nbytes + hp.offsets.nbytes + hp.lengths.nbytes + hp.consts.nbytes
    return {"seconds": statistics.median(ts), "h2d": int(h2d),
            "d2h": int(progs.P * beagle.FITNESS_DTYPE.itemsize)}


def score_population(beagle, torch, pr, stream, flush, steps, warmup, clocks=None,
                     fp64_steps=1, barrier=None, autotune=False):
    """Time one population: FP32c steps (kernel time too), then the FP64 path."""
    ds = beagle.Dataset(pr.X, pr.y)
    dp = beagle.DevicePrograms(pr.programs)
    out = torch.empty((dp.P, 3), dtype=torch.float64, device="cuda")
    tuned = beagle.autotune([(dp, ds, out)])[0] if autotune else None
    if clocks:
        clocks.start()
    beagle.kernel_timing(True)
    beagle.kernel_time()
    ms = timed_steps(lambda: beagle.score_programs(dp, ds, out=out, stream=stream),
                     steps, warmup, stream, flush, barrier)
    clk = clocks.stop() if clocks else None
    beagle.kernel_timing(False)
    kern_ms, kern_n = beagle.kernel_time()
    g32 = beagle.unpack_fitness(out)
    # the cases each program ran (the early exit on invalid programs), on one more call
    # outside the timed region
    counts = torch.zeros(dp.P, dtype=torch.int64, device="cuda")
    beagle.count_cases(counts)
    try:
        beagle.score_programs(dp, ds, out=torch.empty_like(out), stream=stream)
        torch.cuda.synchronize()
    finally:
        beagle.count_cases(None)
    cases_run = counts.cpu().numpy()
    g64, ms64 = None, None
    if fp64_steps > 0:
        ms64 = timed_steps(lambda: beagle.score_programs(dp, ds, out=out, precision="fp64",
                                                         stream=stream),
                           fp64_steps, 0, stream, flush)
        g64 = beagle.unpack_fitness(out)
    # kernel time of the timed steps only (warm-up launches were timed too: drop them)
    kern_avg = kern_ms / max(kern_n, 1) / 1e3
    return {"ds": ds, "dp": dp, "ms": ms, "ms64": ms64, "g32": g32, "g64": g64, "clk": clk,
            "kernel_s": kern_avg, "tuned": tuned, "cases_run": cases_run}


# DRAM bytes (read + write) of one headline fast-pass launch at P = 2,000 programs, measured
# with ncu on the current kernel (dram__bytes_read.sum + dram__bytes_write.sum).
C3_TRAFFIC_P2000 = 167.66e6 + 148.59e6


def headline_traffic(P: int):
    """The headline kernel's DRAM traffic per launch, scaled from the P = 2,000 capture: both
    parts grow with P (input tiles staged once per program group and tile, 44 bytes of
    partials per program and tile)."""
    return {"traffic": C3_TRAFFIC_P2000 * P / 2000.0,
            "traffic_basis": ("dram__bytes_read.sum + dram__bytes_write.sum of one fast-pass "
                              "launch at P = 2,000 (ncu), scaled by P / 2,000")}


def roofline_of(ev, r, pr, sm_mhz, sms, rates):
    """The roofline entry of one timed population (executed operators and cases)."""
    folds = launch_folds(pr.programs.P, pr.N)
    w = case_weights(r.get("cases_run"), pr.N)
    item = (pr.programs, pr.N) if w is None else (pr.programs, pr.N, w)
    return roofline_line(ev, r["kernel_s"], [item], sm_mhz, sms,
                         ev / straight_line_peak(pr.programs, pr.N, rates, folds, w) / 1e9,
                         folds)


def fp32_vs_fp64_path(g32, g64):
    ok = ((g32[2] & 5) == 0) & ((g64[2] & 5) == 0)
    out = {"programs_compared": int(ok.sum())}
    for k, name in ((0, "mse"), (1, "one_minus_r2")):
        a, b = g32[k][ok], g64[k][ok]
        out[name] = {"frac_within_1e-5": float(np.mean(_close(a, b, 1e-5, 1e-7))) if ok.any()
                     else None, "max_rel": _max_rel(a, b)}
    return out


def sub_c1(beagle, synth, torch, stream, flush, args, sm_mhz, sms, rates):
    pr = synth.make_c1()
    r = score_population(beagle, torch, pr, stream, flush, max(200, args.steps),
                         max(3, args.warmup), fp64_steps=5)
    o = oracle_inline(pr.programs, pr.X, pr.y)
    ev = pr.node_evals
    out = {"workload": C1_DESC, "value": ev * len(r["ms"]) / (sum(r["ms"]) / 1e3) / 1e9,
           "unit": "GPoPs", "ms_per_step": statistics.mean(r["ms"]),
           "p50_ms": _pctl(r["ms"], 0.5), "p99_ms": _pctl(r["ms"], 0.99),
           "fp64": {"value": ev / (statistics.median(r["ms64"]) / 1e3) / 1e9},
           "roofline": roofline_of(ev, r, pr, sm_mhz, sms, rates),
           "work": work_info(pr.programs, pr.N, r["cases_run"], statistics.mean(r["ms"])),
           "parity_full_population": parity_gates(r["g32"], r["g64"], o)}
    r["ds"].release()
    return out


def sub_c2(beagle, synth, torch, stream, flush, args, sm_mhz, sms, rates):
    pr = synth.make_c2()
    r = score_population(beagle, torch, pr, stream, flush, max(100, args.steps),
                         max(3, args.warmup), fp64_steps=2)
    idx = np.sort(np.random.default_rng(12).choice(pr.programs.P, 2000, replace=False))
    o = oracle_inline(pr.programs.subset(idx), pr.X, pr.y)
    sel = lambda g: tuple(a[idx] for a in g)  # noqa: E731
    e2e = e2e_host(beagle, pr.programs, r["ds"], stream, 5)
    ev = pr.node_evals
    out = {"workload": C2_DESC, "value": ev * len(r["ms"]) / (sum(r["ms"]) / 1e3) / 1e9,
           "unit": "GPoPs", "ms_per_step": statistics.mean(r["ms"]),
           "p50_ms": _pctl(r["ms"], 0.5), "p99_ms": _pctl(r["ms"], 0.99),
           "fp64": {"value": ev / (statistics.median(r["ms64"]) / 1e3) / 1e9},
           "e2e": {"value": ev / e2e["seconds"] / 1e9, "unit": "GPoPs",
                   "h2d_bytes_per_step": e2e["h2d"], "d2h_bytes_per_step": e2e["d2h"]},
           "roofline": roofline_of(ev, r, pr, sm_mhz, sms, rates),
           "work": work_info(pr.programs, pr.N, r["cases_run"], statistics.mean(r["ms"])),
           "parity_sample": parity_gates(sel(r["g32"]), sel(r["g64"]), o)}
    r["ds"].release()
    return out


def sub_c4(beagle, synth, torch, stream, flush, args, sm_mhz, sms, steps=None, clocks=None):
    pops = synth.make_c4()
    items = []
    for pr in pops:
        ds = beagle.Dataset(pr.X, pr.y)
        dp = beagle.DevicePrograms(pr.programs)
        items.append((dp, ds, torch.empty((dp.P, 3), dtype=torch.float64, device="cuda")))
    ev = sum(pr.node_evals for pr in pops)
    plan = beagle.BatchPlan(items)
    k = steps or max(3, min(10, args.steps))
    warm = max(3, min(args.warmup, 5))
    if clocks:
        clocks.start()
    ms = timed_steps(lambda: plan.launch(stream), k, warm, stream, flush)
    clk = clocks.stop() if clocks else None
    if clk and clk["sm_mhz"]:
        sm_mhz = clk["sm_mhz"]
    # scoring-kernel time: the same batch launched uncaptured (graph replays bypass the
    # library's launch hooks)
    beagle.kernel_timing(True)
    beagle.kernel_time()
    for _ in range(2):
        flush.zero_()
        beagle.score_batch(items, stream=stream)
    torch.cuda.synchronize()
    beagle.kernel_timing(False)
    kern_ms, kern_n = beagle.kernel_time()

    def one_by_one():
        for dp, ds, out in items:
            beagle.score_programs(dp, ds, out=out, stream=stream)
    ms1 = timed_steps(one_by_one, 2, 1, stream, flush)
    # the cases each program ran (early exit on invalid programs), population by population
    # outside the timed region (the case counter follows single-population calls)
    weights = []
    for (dp, ds, out), pr in zip(items, pops):
        counts = torch.zeros(dp.P, dtype=torch.int64, device="cuda")
        beagle.count_cases(counts)
        try:
            beagle.score_programs(dp, ds, out=out, stream=stream)
            torch.cuda.synchronize()
        finally:
            beagle.count_cases(None)
        weights.append(case_weights(counts.cpu().numpy(), pr.N))
    plan.destroy()
    for _, ds, _ in items:
        ds.release()
    kern_s = kern_ms / 1e3 / 2
    return {"workload": C4_DESC, "value": ev * len(ms) / (sum(ms) / 1e3) / 1e9, "unit": "GPoPs",
            "ms_per_step": statistics.mean(ms), "steps": len(ms), "warmup": warm, "clocks": clk,
            "populations": len(pops), "programs": int(sum(p.programs.P for p in pops)),
            "node_evals_per_step": ev, "scoring_launches_per_step": kern_n // 2,
            "one_call_per_population": {"value": ev / (statistics.median(ms1) / 1e3) / 1e9,
                                        "unit": "GPoPs"},
            "executed_case_fraction": float(
                sum(float(w.sum()) * pr.N for w, pr in zip(weights, pops)) /
                max(1.0, sum(float(pr.programs.P) * pr.N for pr in pops))),
            "roofline": roofline_line(ev, kern_s, [(pr.programs, pr.N, w)
                                                   for pr, w in zip(pops, weights)],
                                      sm_mhz or 2070.0, sms)}


def run_headline(args, rank, world, local):
    """The precision workload (50,000 programs x 10^6 cases): FP32c timed, FP64 path, end to
    end through the host-buffer call, the oracle's gates on a 10,000-program sample of the
    timed launch, the CPU baseline, and compact c1/c2/c4 sub-lines."""
    from paper_2607_06731_gb300 import synth
    pr = synth.make_c3(seed=3 + rank, P=args.P or 50_000)
    # the oracle sample runs in a spawned process while the GPU works
    osample = OracleSample(pr, args.parity_sample) if (rank == 0 and args.parity_sample) else None

    import __graft_entry__
    __graft_entry__.build()
    import torch
    from paper_2607_06731_gb300 import beagle
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    stream = torch.cuda.current_stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    clocks = Clocks(local)
    warm = max(3, args.warmup)
    r = score_population(beagle, torch, pr, stream, flush, args.steps, warm, clocks=clocks,
                         fp64_steps=max(1, args.fp64_steps), barrier=barrier,
                         autotune=args.autotune)
    tot_ms = max_over_ranks(sum(r["ms"]), dist, "cuda")
    clk = r["clk"]
    sm_mhz = clk["sm_mhz"] or 2070.0
    e2e = e2e_host(beagle, pr.programs, r["ds"], stream, max(1, args.e2e_steps))
    rates = beagle.measure_op_rates(1.0, stream=stream)
    ev = pr.node_evals
    subs = {}
    if rank == 0 and not args.no_sub:
        subs["c1"] = sub_c1(beagle, synth, torch, stream, flush, args, sm_mhz, sms, rates)
        subs["c2"] = sub_c2(beagle, synth, torch, stream, flush, args, sm_mhz, sms, rates)
        subs["c4"] = sub_c4(beagle, synth, torch, stream, flush, args, sm_mhz, sms)
        subs["c4"].pop("clocks", None)
    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return 0
    parity = None
    if osample is not None:
        o = osample.result()
        sel = lambda g: tuple(a[osample.idx] for a in g)  # noqa: E731
        parity = parity_gates(sel(r["g32"]), sel(r["g64"]), o)
        parity["sample"] = (f"{len(osample.idx)} of {pr.programs.P} programs (seeded) of the "
                            f"timed launch, all {pr.N} cases")
        parity["oracle_seconds"] = float(o["seconds"])
        parity["oracle_threads"] = int(o["threads"])
    cpu = cpu_baseline(pr, args.cpu_seconds)
    ms = r["ms"]
    line = {
        "metric": METRIC,
        "value": ev * args.steps * world / (tot_ms / 1e3) / 1e9,
        "unit": "GPoPs", "n_gpus": world, "steps": args.steps, "warmup": warm,
        "ms_per_step": tot_ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": C3_DESC, "P": pr.programs.P, "N": pr.N, "d": pr.d,
                   "tokens": pr.programs.tokens, "node_evals_per_step": ev,
                   "precision": "fp32-compensated (fp32 ops, compensated fp32 tile sums, fp64 "
                                "cross-tile merge)",
                   "l2": "flushed before every timed step (256 MiB write, outside events)",
                   "parallelism": f"replicas x{world} (independent populations)",
                   "autotuned": r["tuned"], **work_info(pr.programs, pr.N, r["cases_run"], tot_ms / args.steps)},
        "p50_ms": _pctl(ms, 0.5), "p99_ms": _pctl(ms, 0.99),
        "fp64": {"value": ev / (statistics.median(r["ms64"]) / 1e3) / 1e9, "unit": "GPoPs",
                 "ms_per_step": statistics.median(r["ms64"])},
        "fp32c_vs_fp64_speedup": statistics.median(r["ms64"]) / statistics.median(ms),
        "fp32c_vs_fp64_path": fp32_vs_fp64_path(r["g32"], r["g64"]),
        "parity": parity,
        "roofline": {**roofline_of(ev, r, pr, sm_mhz, sms, rates),
                     **headline_traffic(pr.programs.P)},
        "cpu_baseline": cpu,
        "e2e": {"value": ev / e2e["seconds"] / 1e9, "unit": "GPoPs",
                "h2d_bytes_per_step": e2e["h2d"], "d2h_bytes_per_step": e2e["d2h"]},
        "gpu_launches": launches_per_call(pr.programs.P, pr.N) * args.steps,
        "clocks": clk,
        "workloads": subs,
    }
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


def max_over_ranks(value: float, dist, device: str) -> float:
    """The slowest rank's time (the job ends when every rank has finished); identity on 1."""
    if dist is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_gpops(node_evals_per_rank_step: int, steps: int, world: int, ms: float) -> float:
    """Weak scaling: every rank scores its own population of the same size each step."""
    return node_evals_per_rank_step * steps * world / (ms / 1e3) / 1e9


def run_single(args, rank, world, local):
    """One workload on its own line (config.workload names it)."""
    import __graft_entry__
    __graft_entry__.build()
    import torch
    from paper_2607_06731_gb300 import beagle, synth
    torch.cuda.set_device(local)
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    rates = beagle.measure_op_rates(1.0, stream=stream)
    base = {"metric": METRIC, "unit": "GPoPs", "n_gpus": world, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic"}
    clocks = Clocks(local)
    if args.workload == "c5":
        line = run_c5(args, beagle, synth, torch, clocks)
    elif args.workload == "c4":
        sub = sub_c4(beagle, synth, torch, stream, flush, args, None, sms, steps=args.steps,
                     clocks=clocks)
        clk = sub.pop("clocks")
        line = {"value": sub.pop("value"), "steps": sub.pop("steps"),
                "warmup": sub.pop("warmup"), "ms_per_step": sub.pop("ms_per_step"),
                "config": {"workload": sub.pop("workload"), "l2": "256 MiB flush per step"},
                **sub, "gpu_launches": 6 * sub["scoring_launches_per_step"] * args.steps,
                "clocks": clk}
    else:
        maker = {"c1": synth.make_c1, "c2": synth.make_c2, "c3": synth.make_c3}[args.workload]
        pr = maker(P=args.P) if args.P else maker()
        r = score_population(beagle, torch, pr, stream, flush, args.steps, max(3, args.warmup),
                             clocks=clocks, fp64_steps=args.fp64_steps, autotune=args.autotune)
        ev = pr.node_evals
        sm_mhz = r["clk"]["sm_mhz"] or 2070.0
        desc = {"c1": C1_DESC, "c2": C2_DESC, "c3": C3_DESC}[args.workload]
        e2e = e2e_host(beagle, pr.programs, r["ds"], stream, max(1, args.e2e_steps))
        line = {"value": ev * len(r["ms"]) / (sum(r["ms"]) / 1e3) / 1e9, "steps": args.steps,
                "warmup": max(3, args.warmup), "ms_per_step": statistics.mean(r["ms"]),
                "p50_ms": _pctl(r["ms"], 0.5), "p99_ms": _pctl(r["ms"], 0.99),
                "config": {"workload": desc, "P": pr.programs.P, "N": pr.N, "d": pr.d,
                           "node_evals_per_step": ev, "autotuned": r["tuned"],
                           "l2": "256 MiB flush before every step",
                           **work_info(pr.programs, pr.N, r["cases_run"], statistics.mean(r["ms"]))},
                "fp64": ({"value": ev / (statistics.median(r["ms64"]) / 1e3) / 1e9}
                         if r["ms64"] else None),
                "fp32c_vs_fp64_path": fp32_vs_fp64_path(r["g32"], r["g64"]) if r["g64"] else None,
                "roofline": roofline_of(ev, r, pr, sm_mhz, sms, rates),
                "e2e": {"value": ev / e2e["seconds"] / 1e9, "unit": "GPoPs",
                        "h2d_bytes_per_step": e2e["h2d"], "d2h_bytes_per_step": e2e["d2h"]},
                "cpu_baseline": cpu_baseline(pr, args.cpu_seconds),
                "gpu_launches": launches_per_call(pr.programs.P, pr.N) * args.steps,
                "clocks": r["clk"]}
        r["ds"].release()
    if rank == 0:
        print(json.dumps({**base, **line}), flush=True)
    return 0


def run_c5(args, beagle, synth, torch, clocks):
    """Serving: 16 evolutionary runs, each with a resident dataset (N log-U[512, 65536], d
    U{1..10}), drive one server in a closed loop -- a run submits its next generation (P
    log-U[1e4, 5e5] programs of length U{8..200}) only after it has received the previous
    one's fitness, after an exponentially distributed think time. The same fixed set of
    requests (args.requests in all, spread over the runs) is served at every load level: no
    think time (saturation: the capacity), then mean think times that put the device at about
    0.9x and 0.5x of that capacity. Per level: GPoPs, p50 / p99 latency (submit to result)
    raw and per node evaluation, time queued before admission, kernel launches. Request
    populations are slices of one 100k-program population per input count d, generated before
    timing."""
    import threading
    runs = synth.make_serving_runs()
    nruns = len(runs)
    dsets = [beagle.Dataset(r["X"], r["y"]) for r in runs]
    pools = {}
    for r in runs:
        if r["d"] not in pools:
            pools[r["d"]] = synth.gen_programs(np.random.default_rng([5, 3, r["d"]]), 100_000,
                                               8, 200, r["d"])
    rng = np.random.default_rng([5, 4])
    per_run = [[] for _ in range(nruns)]
    for k in range(args.requests):
        run = k % nruns
        pool = pools[runs[run]["d"]]
        P = int(np.exp(rng.uniform(np.log(1e4), np.log(5e5))))
        start = int(rng.integers(pool.P))
        progs = pool.subset((start + np.arange(P)) % pool.P)
        per_run[run].append((progs, int(progs.lengths.sum()) * runs[run]["N"]))
    total_evals = sum(e for rr in per_run for _, e in rr)

    def level(think_mean_s, seed):
        srv = beagle.Server()
        recs, errs = [], []
        lock = threading.Lock()

        def client(i):
            r = np.random.default_rng([seed, i])
            try:
                for progs, ev in per_run[i]:
                    if think_mean_s > 0:
                        time.sleep(r.exponential(think_mean_s))
                    t = srv.submit(progs, dsets[i])
                    srv.wait(t)
                    with lock:
                        recs.append((t, ev))
            except Exception as e:   # reported below
                errs.append(e)
        t0 = time.perf_counter()
        th = [threading.Thread(target=client, args=(i,)) for i in range(nruns)]
        for t in th:
            t.start()
        for t in th:
            t.join()
        wall = time.perf_counter() - t0
        if errs:
            raise errs[0]
        lat = np.array([srv.timing(t)["latency_us"] for t, _ in recs])
        que = np.array([srv.timing(t)["queue_us"] for t, _ in recs])
        evs = np.array([ev for _, ev in recs], np.float64)
        st = srv.stats()
        srv.destroy()
        per = lat * 1e3 / evs     # ns per node evaluation
        return {"requests": len(recs), "think_mean_ms": think_mean_s * 1e3,
                "wall_s": wall, "gpops": float(evs.sum() / wall / 1e9),
                "p50_ms": float(np.percentile(lat, 50) / 1e3),
                "p99_ms": float(np.percentile(lat, 99) / 1e3),
                "max_ms": float(lat.max() / 1e3),
                "p50_ns_per_node_eval": float(np.percentile(per, 50)),
                "p99_ns_per_node_eval": float(np.percentile(per, 99)),
                "queue_p50_ms": float(np.percentile(que, 50) / 1e3),
                "queue_p99_ms": float(np.percentile(que, 99) / 1e3),
                "launches": st["launches"], "peak_gb": st["peak_bytes"] / 1e9,
                "budget_gb": st["budget_bytes"] / 1e9}

    # warm-up: one request per run
    srv = beagle.Server()
    for i in range(nruns):
        srv.wait(srv.submit(per_run[i][0][0], dsets[i]))
    srv.destroy()
    clocks.start()
    sat = level(0.0, 1)
    cap_rps = sat["requests"] / sat["wall_s"]
    levels = {"saturated": sat}
    for f in (0.9, 0.5):
        # closed loop: each run's cycle is think + response; about f of the capacity when the
        # think time is nruns / (f * capacity) less the saturated cycle's response share
        think = max(0.0, nruns / (f * cap_rps) - nruns / cap_rps)
        lv = level(think, int(f * 10))
        lv["utilisation"] = lv["gpops"] / sat["gpops"]
        levels[f"{f}x"] = lv
    clk = clocks.stop()
    ex_run = 0
    pr = synth.Problem("c5-sample", per_run[ex_run][0][0], runs[ex_run]["X"], runs[ex_run]["y"], {})
    for ds in dsets:
        ds.release()
    nreq = args.requests
    return {"value": sat["gpops"], "steps": nreq, "warmup": nruns,
            "ms_per_step": sat["wall_s"] / nreq * 1e3,
            "p50_ms": sat["p50_ms"], "p99_ms": sat["p99_ms"],
            "config": {"workload": "c5-serving: 16 runs with resident datasets (N log-U[512,"
                                   "65536], d U{1..10}), closed loop, Poisson think times; "
                                   "requests P log-U[1e4,5e5], L U{8..200}",
                       "requests_per_level": nreq, "node_evals_per_level": total_evals,
                       "l2": "inputs larger than L2 per request"},
            "levels": levels,
            "e2e": {"value": sat["gpops"], "unit": "GPoPs",
                    "h2d_bytes_per_step": int(np.mean([p.ops.nbytes * 5 + p.P * 12
                                                       for rr in per_run for p, _ in rr])),
                    "d2h_bytes_per_step": int(np.mean([p.P * 24 for rr in per_run
                                                       for p, _ in rr]))},
            "roofline": None,
            "cpu_baseline": cpu_baseline(pr, args.cpu_seconds),
            "gpu_launches": sum(lv["launches"] for lv in levels.values()), "clocks": clk}


# Programs that repeat one interpreter handler n times (after a first leaf), for the handler
# profile: each (name, n) is one scoring launch of HANDLER_P programs on HANDLER_N cases.
HANDLER_P, HANDLER_N = 2048, 1024


def handler_programs():
    from paper_2607_06731_gb300 import synth as S
    L0, L1, C = S.LOAD0, S.LOAD0 + 1, S.CONST

    def rep(body, n, suffix=()):
        return [(L0, 0.0)] + list(body) * n + list(suffix)
    return {
        "ADDX": lambda n: rep([(L1, 0.0), (S.ADD, 0.0)], n),
        "MULX": lambda n: rep([(L1, 0.0), (S.MUL, 0.0)], n),
        "ADDC": lambda n: rep([(C, 0.5), (S.ADD, 0.0)], n),
        "PDIVX": lambda n: rep([(L1, 0.0), (S.PDIV, 0.0)], n),
        "PUSHX+ADD": lambda n: rep([(L1, 0.0)], n, [(S.ADD, 0.0)] * n),
        "PUSHX+PDIV": lambda n: rep([(L1, 0.0)], n, [(S.PDIV, 0.0)] * n),
        "DUP+MUL": lambda n: rep([(S.DUP, 0.0), (S.MUL, 0.0)], n),
        "SIN": lambda n: rep([(S.SIN, 0.0)], n),
        "COS": lambda n: rep([(S.COS, 0.0)], n),
        "EXP": lambda n: rep([(S.EXP, 0.0)], n),
        "PLOG": lambda n: rep([(S.PLOG, 0.0)], n),
        "PSQRT": lambda n: rep([(S.PSQRT, 0.0)], n),
        "SQUARE": lambda n: rep([(S.SQUARE, 0.0)], n),
    }


def run_handlers(args):
    """One launch per (handler, n) for n = 8 and 15; prints each launch's interpreter steps
    (tokens after leaf + binary fusion, plus END, per 128-case pass, over all programs). Under
    ncu, (instructions(15) - instructions(8)) / (steps(15) - steps(8)) is the handler's cost.
    The early exit on invalid programs is off: a chain of 15 exps or squares overflows, and
    every case must still run for the count to hold."""
    import torch
    from paper_2607_06731_gb300 import beagle, synth as S
    X = np.random.default_rng(0).uniform(0.5, 1.5, (3, HANDLER_N)).astype(np.float32)
    y = (X[0] + X[1]).astype(np.float32)
    ds = beagle.Dataset(X, y)
    beagle.set_launch_config(cases_per_lane=4, tile=512, keep_order=1)
    beagle.set_invalid_early_exit(False)
    lines = []
    try:
        for name, mk in handler_programs().items():
            for n in (8, 15):
                toks = mk(n)
                dp = beagle.DevicePrograms(S.from_token_lists([toks] * HANDLER_P))
                beagle.score_programs(dp, ds)
                torch.cuda.synchronize()
                ops = [t[0] for t in toks]
                leaf = [o == S.CONST or S.LOAD0 <= o < S.LOAD0 + 16 for o in ops]
                fused = sum(1 for i in range(len(ops) - 1)
                            if leaf[i] and ops[i + 1] in (S.ADD, S.SUB, S.MUL, S.PDIV))
                steps = (len(ops) - fused + 1) * HANDLER_P * (HANDLER_N // 128)
                lines.append({"handler": name, "n": n, "steps": steps})
                print(json.dumps(lines[-1]), flush=True)
    finally:
        beagle.set_invalid_early_exit(True)
        beagle.reset_launch_config()
        ds.release()
    return 0


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if args.workload == "handlers":
        return run_handlers(args)
    if args.workload == "headline":
        return run_headline(args, rank, world, local)
    return run_single(args, rank, world, local)


if __name__ == "__main__":
    sys.exit(main())
