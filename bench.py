#!/usr/bin/env python3
"""Population fitness scoring benchmark: GPoPs (program-node evaluations per second).

One step = one beagle_score call over the whole population of the workload: every program
interpreted on every fitness case and reduced to its MSE and 1 - r^2 (Beagle tutorial,
Section 2.4). Default workload: P = 100,000 random postfix programs (length U{16..128},
d = 5 inputs), N = 1,024 fitness cases, X ~ U[-3, 3], y = a random 20-node expression plus
N(0, 0.01) noise, on the FP32-compensated path. Inputs are resident in HBM before timing;
L2 is flushed (a 256 MiB write) before every timed step, outside the timed events.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun each rank scores its own population (seed + rank) on its own GPU with no
collective on the data path (weak scaling); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "GPoPs (node-evals/s) FP32-compensated vs plain FP64 at ≤1e-5 rel err; p50/p99"
# kernels one scoring call launches: length order, persistent scoring kernel, fp64 finalize
LAUNCHES_PER_CALL = 3
WORKLOAD = ("c2-population-100k: P=100000 programs, length U{16..128}, d=5, N=1024 cases, "
            "X~U[-3,3], y=20-node expression + N(0,0.01) noise; MSE and 1-R^2")


def parse():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--fp64-steps", type=int, default=3)
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--P", type=int, default=100_000)
    ap.add_argument("--cpu-seconds", type=float, default=10.0,
                    help="target wall time of the CPU oracle sample")
    ap.add_argument("--workload", choices=["c1", "c2", "c3", "c4", "c5"], default="c2",
                    help="c2: one 100k population (default, the headline line); c1: 1024 "
                         "programs x 1024 cases (the oracle-sized case); c3: 50k "
                         "programs x 1e6 cases, d=10 (precision); c4: 64 ragged populations "
                         "in one graph-captured batch; c5: serving loop under Poisson load")
    ap.add_argument("--requests", type=int, default=32,
                    help="c5: requests per load level")
    ap.add_argument("--autotune", action="store_true",
                    help="c1/c3/c4: let beagle_autotune pick the launch shape before timing")
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


# DRAM traffic of the scoring kernel from an ncu capture (dram__bytes_read.sum +
# dram__bytes_write.sum of the P = 20,000 case, scaled by 5 to a full launch: traffic is per
# program), valid only for the kernel sources it was taken on (profiles/ has the capture).
TRAFFIC_CAPTURE = {
    "sources_sha256": "538eac4a4b5dbd2428a72dee4eef4f0f14249baab51ae1a2f9cb8876c8e594f1",
    "bytes_per_launch": 39_307_520,   # (7,747,584 read + 113,920 written) x 5
}


# the files that define the scoring kernel's device code
KERNEL_SOURCES = ("common.cuh", "interp_ptx.cuh", "interp_ptx8.cuh", "score.cuh",
                  "score_kernels.cu", "transcend.cuh")


def kernel_sources_sha256(d=None):
    import hashlib
    d = d or os.path.join(ROOT, "paper_2607_06731_gb300", "csrc")
    h = hashlib.sha256()
    for name in KERNEL_SOURCES:
        h.update(name.encode())
        h.update(open(os.path.join(d, name), "rb").read())
    return h.hexdigest()


def captured_traffic():
    cap = TRAFFIC_CAPTURE
    if cap["sources_sha256"] and cap["sources_sha256"] == kernel_sources_sha256():
        return cap["bytes_per_launch"]
    return None


# Issue roofline from unit counts and clocks. Instructions per evaluation of each operator as
# implemented (validity check included), total and per pipe: ncu counters
# (smsp__inst_executed[_pipe_fma|_alu|_xu].sum) of the straight-line operator microbenchmark
# (beagle_measure_op_rates) divided by its evaluations (profiles/op_instruction_mix.md). Peak
# rates per SM per cycle (ncu .peak_sustained): issue 4 warp instructions, FMA pipe 4, ALU 2,
# XU 1. Valid while the sources that define the operators hash as below.
OP_INSTR = {
    "sources_sha256": "f6dc884c9294e922d0cc50a7e86c3506fe88d9afdfd81be49e948521fe9b7ac1",
    "per_sm_cycle": {"all": 4, "fma": 4, "alu": 2, "xu": 1},
    "per_eval": {   # opcode: (all, fma, alu, xu)
        1: (1.875, 1.0, 0.75, 0.0), 2: (1.875, 1.0, 0.75, 0.0), 3: (1.875, 1.0, 0.75, 0.0),
        4: (8.876, 5.001, 2.75, 1.0), 5: (28.502, 17.001, 7.0, 0.0),
        6: (29.502, 17.251, 7.75, 0.0), 7: (9.126, 6.126, 1.625, 1.0),
        8: (23.502, 16.126, 7.0, 0.0), 9: (12.376, 5.001, 3.0, 1.0),
        10: (1.875, 1.0, 0.5, 0.0),
    },
}
OP_SOURCES = ("common.cuh", "measure.cu", "score.cuh", "transcend.cuh")


def issue_roofline(progs_list, sm_mhz: float, sms: int = 152):
    """Time the op work of the populations (list of (programs, N)) needs at the issue and pipe
    rates; leaves and stack moves are free. None if the operator table is stale."""
    import hashlib
    d = os.path.join(ROOT, "paper_2607_06731_gb300", "csrc")
    h = hashlib.sha256()
    for name in OP_SOURCES:
        h.update(name.encode())
        h.update(open(os.path.join(d, name), "rb").read())
    if h.hexdigest() != OP_INSTR["sources_sha256"]:
        return None
    pipes = ("all", "fma", "alu", "xu")
    inst = dict.fromkeys(pipes, 0.0)
    for progs, N in progs_list:
        counts = np.bincount(progs.ops, minlength=64).astype(np.float64)
        for op, per in OP_INSTR["per_eval"].items():
            for k, v in zip(pipes, per):
                inst[k] += counts[op] * N * v
    f = sm_mhz * 1e6
    t = {k: inst[k] / (OP_INSTR["per_sm_cycle"][k] * 32 * sms * f) for k in pipes}
    bind = max(t, key=t.get)
    return {"seconds": t[bind], "binding": "issue" if bind == "all" else bind + " pipe",
            "per_pipe_ms": {k: v * 1e3 for k, v in t.items()}}


def roofline_peak(progs, N, rates):
    """ALU-issue roofline: the time straight-line compiled code would need for this op mix,
    every operator at its measured throughput (validity check included), leaves free."""
    counts = np.bincount(progs.ops, minlength=64).astype(np.float64)
    t = 0.0
    for op, r in rates.items():
        t += counts[op] * N / r
    return t


def cpu_baseline(pr, seconds: float, threads: int = 0):
    """Time the oracle (FP64, as it stands) on a seeded sample of the population."""
    import oracle
    oracle.build()
    rng = np.random.default_rng(1234)
    mean_len = float(pr.programs.lengths.mean())
    n = int(min(pr.programs.P, max(2, min(200, 2e8 / (mean_len * pr.N)))))
    idx = rng.choice(pr.programs.P, n, replace=False)
    sub = pr.programs.subset(idx)
    t0 = time.perf_counter()
    oracle.score_programs(sub, pr.X, pr.y, "fp64", nthreads=threads)
    dt = max(time.perf_counter() - t0, 1e-6)
    n2 = int(min(pr.programs.P, max(n, n * seconds / dt)))
    idx = rng.choice(pr.programs.P, n2, replace=False)
    sub = pr.programs.subset(idx)
    t0 = time.perf_counter()
    oracle.score_programs(sub, pr.X, pr.y, "fp64", nthreads=threads)
    dt = time.perf_counter() - t0
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


def aggregation_error(beagle, synth, progs, pr, ds, fp32, n=2000):
    """Relative error of the FP32c fitness against plain fp64 sums of the same per-case fp32
    outputs, over a seeded sample of valid, non-degenerate programs."""
    import torch
    rng = np.random.default_rng(7)
    idx = np.sort(rng.choice(progs.P, min(n, progs.P), replace=False))
    dp = beagle.DevicePrograms(progs.subset(idx))
    outs, _ = beagle.eval_programs(dp, ds)
    f = outs.double().cpu().numpy()
    torch.cuda.synchronize()
    y = pr.y.astype(np.float64)
    with np.errstate(invalid="ignore", divide="ignore", over="ignore"):   # invalid programs
        mse = ((f - y) ** 2).mean(axis=1)
        fc = f - f.mean(axis=1, keepdims=True)
        yc = y - y.mean()
        r = (fc * yc).sum(axis=1) / np.sqrt((fc * fc).sum(axis=1) * (yc * yc).sum())
        omr = 1.0 - r * r
    ok = (fp32[2][idx] == 0) & np.isfinite(mse) & np.isfinite(omr)
    out = {"programs_compared": int(ok.sum())}
    for name, ref, got in (("mse", mse, fp32[0][idx]), ("one_minus_r2", omr, fp32[1][idx])):
        a, b = got[ok], ref[ok]
        err = np.abs(a - b)
        rel = err / np.maximum(np.abs(b), 1e-300)
        out[name] = {"frac_within_1e-5": float(np.mean(err <= np.maximum(1e-5 * np.abs(b),
                                                                           1e-7))),
                     "max_rel": float(rel.max()) if len(rel) else None,
                     "median_rel": float(np.median(rel)) if len(rel) else None}
    return out


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


def run_reference(args, rank, world):
    """The oracle timed as the reference arm: each step scores a bounded seeded sample."""
    if rank != 0:
        return 0
    from paper_2607_06731_gb300 import synth
    import oracle
    oracle.build()
    pr = synth.make_c2(P=args.P)
    rng = np.random.default_rng(99)
    n = 200
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
            "config": {"workload": WORKLOAD, "P": pr.programs.P, "N": pr.N, "d": pr.d,
                       "sample_programs": n},
            "cpu_baseline": {"value": value, "unit": "GPoPs", "cores": oracle.threads(),
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "GPoPs", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------------------- c3 / c4 / c5
def _timed_steps(step, steps, warmup, stream, flush):
    import torch
    for _ in range(max(3, warmup)):
        flush.zero_()
        step()
    torch.cuda.synchronize()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(steps)]
    for a, b in evs:
        flush.zero_()
        a.record(stream)
        step()
        b.record(stream)
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in evs]


def _pctl(v, q):
    v = sorted(v)
    return v[min(len(v) - 1, int(round(q * (len(v) - 1))))] if v else None


def run_other_workload(args, rank, world, local):
    """Secondary workloads, each printing its own JSON line (config.workload names it)."""
    import __graft_entry__
    __graft_entry__.build()
    import torch
    from paper_2607_06731_gb300 import beagle, synth
    torch.cuda.set_device(local)
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    rates = beagle.measure_op_rates(1.0, stream=stream)
    clocks = Clocks(local)
    base = {"metric": METRIC, "unit": "GPoPs", "n_gpus": world, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic"}
    if args.workload in ("c1", "c3"):
        line = _run_c3(args, beagle, synth, torch, stream, flush, rates, clocks, args.workload)
    elif args.workload == "c4":
        line = _run_c4(args, beagle, synth, torch, stream, flush, rates, clocks)
    else:
        line = _run_c5(args, beagle, synth, torch, stream, rates, clocks)
    if rank == 0:
        print(json.dumps({**base, **line}), flush=True)
    return 0


C1_DESC = ("c1-small-1024: P=1024 programs, length U{8..32}, d=2, N=1024 cases, X~U[-3,3], "
           "y = x0 sin(x1) + x0^2/2")
C3_DESC = ("c3-precision-1m: P=50000 programs, length U{16..64}, d=10, N=1000000 cases, "
           "X~N(0,1), y RMS 1e3 + N(0,1)")


def _run_c3(args, beagle, synth, torch, stream, flush, rates, clocks, which="c3"):
    """One population on one dataset, FP32-compensated and plain FP64 paths, the error of the
    first against the second: the precision workload (50,000 programs, length U{16..64}, on
    1e6 cases, d = 10, y of RMS 1e3) or the small oracle-sized one (c1)."""
    pr = synth.make_c3() if which == "c3" else synth.make_c1()
    ds = beagle.Dataset(pr.X, pr.y)
    dp = beagle.DevicePrograms(pr.programs)
    out = torch.empty((dp.P, 3), dtype=torch.float64, device="cuda")
    tuned = beagle.autotune([(dp, ds, out)])[0] if args.autotune else None
    clocks.start()
    beagle.kernel_timing(True)
    beagle.kernel_time()
    ms = _timed_steps(lambda: beagle.score_programs(dp, ds, out=out, stream=stream),
                      args.steps, args.warmup, stream, flush)
    clk = clocks.stop()
    beagle.kernel_timing(False)
    kern_ms, kern_n = beagle.kernel_time()
    f32 = beagle.unpack_fitness(out)
    ms64 = _timed_steps(lambda: beagle.score_programs(dp, ds, out=out, precision="fp64",
                                                      stream=stream),
                        max(1, args.fp64_steps), 0, stream, flush)
    f64 = beagle.unpack_fitness(out)
    ok = ((f32[2] & 5) == 0) & ((f64[2] & 5) == 0)
    err = {}
    for k, name in ((0, "mse"), (1, "one_minus_r2")):
        a, b = f32[k][ok], f64[k][ok]
        rel = np.abs(a - b) / np.maximum(np.abs(b), 1e-300)
        err[name] = {"frac_within_1e-5": float(np.mean(np.abs(a - b) <=
                                                        np.maximum(1e-5 * np.abs(b), 1e-7))),
                     "median_rel": float(np.median(rel)), "max_rel": float(rel.max())}
    ev = pr.node_evals
    kern_s = kern_ms / max(kern_n, 1) / 1e3
    peak_straight = ev / roofline_peak(pr.programs, pr.N, rates) / 1e9
    issue = issue_roofline([(pr.programs, pr.N)], clk["sm_mhz"] or 2070.0)
    peak = ev / issue["seconds"] / 1e9 if issue else peak_straight
    return {"value": ev * len(ms) / (sum(ms) / 1e3) / 1e9, "steps": len(ms),
            "warmup": max(3, args.warmup), "ms_per_step": statistics.mean(ms),
            "p50_ms": _pctl(ms, 0.5), "p99_ms": _pctl(ms, 0.99),
            "config": {"workload": C3_DESC if which == "c3" else C1_DESC,
                       "P": dp.P, "N": pr.N, "d": pr.d, "node_evals_per_step": ev,
                       "l2": "256 MiB flush before every step", "autotuned": tuned},
            "fp64": {"value": ev / (statistics.median(ms64) / 1e3) / 1e9, "unit": "GPoPs",
                     "ms_per_step": statistics.median(ms64)},
            "fp32c_error_vs_fp64_path": {"programs_compared": int(ok.sum()), **err},
            "roofline": {"bound": "alu", "achieved": ev / kern_s / 1e9, "peak": peak,
                         "unit": "GPoPs", "frac": ev / kern_s / 1e9 / peak, "traffic": None,
                         "peak_basis": ("issue roofline, binding: " + issue["binding"])
                                       if issue else "straight-line per-op throughput",
                         "peak_straight_line_ops": peak_straight},
            "cpu_baseline": cpu_baseline(pr, args.cpu_seconds),
            "gpu_launches": LAUNCHES_PER_CALL * len(ms), "clocks": clk}


def _run_c4(args, beagle, synth, torch, stream, flush, rates, clocks):
    """64 ragged populations (P log-U[1e3, 2e5], L U{4..256}, N log-U[256, 1e5], d U{1..10}),
    each with its own resident dataset, scored in one graph-captured persistent batch; the
    same populations scored one call each for comparison."""
    pops = synth.make_c4()
    items = []
    for pr in pops:
        ds = beagle.Dataset(pr.X, pr.y)
        dp = beagle.DevicePrograms(pr.programs)
        items.append((dp, ds, torch.empty((dp.P, 3), dtype=torch.float64, device="cuda")))
    ev = sum(pr.node_evals for pr in pops)
    tuned = beagle.autotune(items)[0] if args.autotune else None
    plan = beagle.BatchPlan(items)
    clocks.start()
    ms = _timed_steps(lambda: plan.launch(stream), args.steps, args.warmup, stream, flush)
    clk = clocks.stop()
    # kernel time of the scoring kernel: the same batch launched uncaptured (graph replays
    # bypass the library's launch hooks)
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
    ms1 = _timed_steps(one_by_one, max(1, min(3, args.steps)), 1, stream, flush)
    t_roof = sum(roofline_peak(pr.programs, pr.N, rates) for pr in pops)
    issue = issue_roofline([(pr.programs, pr.N) for pr in pops], clk["sm_mhz"] or 2070.0)
    if issue:
        t_roof = issue["seconds"]
    # scoring launches per batch (the batch is cut by input width), each with its length
    # order and finalize kernels
    launches_per_plan = (kern_n // 2) * LAUNCHES_PER_CALL
    kern_s = kern_ms / 1e3 / 2                   # scoring-kernel time per batch (all launches)
    big = max(pops, key=lambda p: p.node_evals)
    return {"value": ev * len(ms) / (sum(ms) / 1e3) / 1e9, "steps": len(ms),
            "warmup": max(3, args.warmup), "ms_per_step": statistics.mean(ms),
            "p50_ms": _pctl(ms, 0.5), "p99_ms": _pctl(ms, 0.99),
            "config": {"workload": "c4-ragged-64: 64 populations, P log-U[1e3,2e5], "
                                   "L U{4..256}, N log-U[256,1e5], d U{1..10}, one dataset "
                                   "each; one graph-captured batch per step",
                       "populations": len(pops), "programs": int(sum(p.programs.P for p in pops)),
                       "node_evals_per_step": ev, "autotuned": tuned,
                       "l2": "256 MiB flush before every step"},
            "one_call_per_population": {"value": ev / (statistics.median(ms1) / 1e3) / 1e9,
                                        "unit": "GPoPs", "ms_per_step": statistics.median(ms1)},
            "roofline": {"bound": "alu", "achieved": ev / kern_s / 1e9 if kern_s else None,
                         "peak": ev / t_roof / 1e9, "unit": "GPoPs",
                         "frac": (ev / kern_s / 1e9) / (ev / t_roof / 1e9) if kern_s else None,
                         "traffic": None, "kernel_launches_timed": kern_n,
                         "peak_basis": ("issue roofline, binding: " + issue["binding"])
                                       if issue else "straight-line per-op throughput"},
            "cpu_baseline": cpu_baseline(big, args.cpu_seconds),
            "gpu_launches": launches_per_plan * len(ms), "clocks": clk}


def _run_c5(args, beagle, synth, torch, stream, rates, clocks):
    """Serving: 16 evolutionary runs with resident datasets submit generations (P log-U[1e4,
    5e5], L U{8..200}) to one server; first at once (capacity), then as Poisson arrivals at
    0.5x, 0.9x and 1.2x of that capacity. Reports GPoPs and p50 / p99 latency per level.
    Request populations are slices of one 100k-program population per input count d (cycled
    where a request asks for more), generated before timing."""
    runs = synth.make_serving_runs()
    dsets = [beagle.Dataset(r["X"], r["y"]) for r in runs]
    pools = {}
    for r in runs:
        if r["d"] not in pools:
            pools[r["d"]] = synth.gen_programs(np.random.default_rng([5, 3, r["d"]]), 100_000,
                                               8, 200, r["d"])
    rng = np.random.default_rng([5, 4])

    def make_requests(n):
        reqs = []
        for k in range(n):
            run = int(rng.integers(len(runs)))
            pool = pools[runs[run]["d"]]
            P = int(np.exp(rng.uniform(np.log(1e4), np.log(5e5))))
            start = int(rng.integers(pool.P))
            progs = pool.subset((start + np.arange(P)) % pool.P)
            reqs.append((run, progs, int(progs.lengths.sum()) * runs[run]["N"]))
        return reqs

    def serve(reqs, rate_rps):
        srv = beagle.Server()
        res = []
        t0 = time.perf_counter()

        tickets = []
        arr = np.cumsum(rng.exponential(1.0 / rate_rps, len(reqs))) if rate_rps else None
        for k, (run, progs, _) in enumerate(reqs):
            if arr is not None:
                dt = t0 + arr[k] - time.perf_counter()
                if dt > 0:
                    time.sleep(dt)
            tickets.append(srv.submit(progs, dsets[run]))
        for t in tickets:        # latency is measured by the server (submit to result)
            res.append(srv.wait(t))
        wall = time.perf_counter() - t0
        st = srv.stats()
        srv.destroy()
        return wall, st

    warm = make_requests(4)
    serve(warm, 0)
    reqs = make_requests(args.requests)
    ev = sum(r[2] for r in reqs)
    clocks.start()
    wall, st = serve(reqs, 0)
    cap_rps = len(reqs) / wall
    levels = {}
    for f in (0.5, 0.9, 1.2):
        reqs_f = make_requests(args.requests)
        w, s2 = serve(reqs_f, f * cap_rps)
        levels[f"{f}x"] = {"offered_rps": f * cap_rps, "gpops": s2["gpops"],
                           "p50_ms": s2["p50_us"] / 1e3, "p99_ms": s2["p99_us"] / 1e3,
                           "max_ms": s2["max_us"] / 1e3, "launches": s2["launches"],
                           "peak_gb": s2["peak_bytes"] / 1e9}
    clk = clocks.stop()
    ex = make_requests(1)[0]
    pr = synth.Problem("c5-sample", ex[1], runs[ex[0]]["X"], runs[ex[0]]["y"], {})
    return {"value": st["gpops"], "steps": len(reqs), "warmup": len(warm),
            "ms_per_step": wall / len(reqs) * 1e3,
            "p50_ms": st["p50_us"] / 1e3, "p99_ms": st["p99_us"] / 1e3,
            "config": {"workload": "c5-serving: 16 runs with resident datasets (N log-U[512,"
                                   "65536], d U{1..10}); requests P log-U[1e4,5e5], "
                                   "L U{8..200}; closed loop, then Poisson at 0.5/0.9/1.2x",
                       "requests_per_level": len(reqs), "node_evals_closed_loop": ev,
                       "budget_bytes": st["budget_bytes"],
                       "l2": "inputs larger than L2 per request"},
            "closed_loop": {"requests_per_s": cap_rps, "launches": st["launches"],
                            "peak_gb": st["peak_bytes"] / 1e9},
            "poisson": levels,
            "e2e": {"value": st["gpops"], "unit": "GPoPs",
                    "h2d_bytes_per_step": int(np.mean([r[1].ops.nbytes * 5 + r[1].P * 12
                                                       for r in reqs])),
                    "d2h_bytes_per_step": int(np.mean([r[1].P * 24 for r in reqs]))},
            "roofline": None,
            "cpu_baseline": cpu_baseline(pr, args.cpu_seconds),
            "gpu_launches": st["launches"] * LAUNCHES_PER_CALL, "clocks": clk}


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.impl == "reference":
        return run_reference(args, rank, world)

    if args.workload != "c2":
        return run_other_workload(args, rank, world, local)

    import __graft_entry__
    __graft_entry__.build()
    import torch
    from paper_2607_06731_gb300 import beagle, synth

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    pr = synth.make_c2(seed=2 + rank, P=args.P)
    progs = pr.programs
    node_evals = pr.node_evals
    ds = beagle.Dataset(pr.X, pr.y)
    dp = beagle.DevicePrograms(progs)
    out = torch.empty((progs.P, 3), dtype=torch.float64, device="cuda")
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()

    def step(precision="fp32c"):
        beagle.score_programs(dp, ds, out=out, precision=precision, stream=stream)

    # W untimed warm-up steps, continued until a second of work has run: the first second in a
    # fresh process runs a few per cent slower while the clocks settle.
    warm = 0
    t_warm = time.perf_counter()
    while warm < max(3, args.warmup) or time.perf_counter() - t_warm < 1.0:
        flush.zero_()
        step()
        warm += 1
        if warm % 16 == 0:
            torch.cuda.synchronize()
    barrier()
    clocks = Clocks(local)
    clocks.start()
    beagle.kernel_timing(True)
    beagle.kernel_time()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    barrier()
    for a, b in evs:
        flush.zero_()
        a.record(stream)
        step()
        b.record(stream)
    barrier()
    clk = clocks.stop()
    beagle.kernel_timing(False)
    kern_ms, kern_launches = beagle.kernel_time()
    step_ms = [a.elapsed_time(b) for a, b in evs]
    tot_ms = sum(step_ms)
    tot_ms = max_over_ranks(tot_ms, dist, "cuda")
    fp32 = beagle.unpack_fitness(out)

    # plain FP64 path (same workload, fewer steps)
    step("fp64")
    torch.cuda.synchronize()
    f64_ms = []
    for _ in range(args.fp64_steps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        step("fp64")
        b.record(stream)
        torch.cuda.synchronize()
        f64_ms.append(a.elapsed_time(b))
    fp64 = beagle.unpack_fitness(out)

    # relative error of FP32c against the FP64 path (valid programs in both)
    ok = ((fp32[2] & 5) == 0) & ((fp64[2] & 5) == 0)
    rel = np.abs(fp32[0][ok] - fp64[0][ok]) / np.maximum(np.abs(fp64[0][ok]), 1e-300)
    within = (np.abs(fp32[0][ok] - fp64[0][ok]) <= np.maximum(1e-5 * np.abs(fp64[0][ok]), 1e-7))

    # The aggregation alone: the FP32c path's fitness against plain fp64 sums (numpy) of the
    # same per-case fp32 outputs (beagle_eval), on a seeded sample of programs.
    agg = aggregation_error(beagle, synth, progs, pr, ds, fp32)

    # end to end through the host-buffer C-ABI call (copies inside the timed region)
    host = synth.Programs(*(np.ascontiguousarray(a) for a in
                            (progs.ops, progs.offsets, progs.lengths, progs.consts)))
    pinned = [torch.from_numpy(a).pin_memory() for a in
              (host.ops, host.offsets, host.lengths, host.consts)]
    hp = synth.Programs(*(t.numpy() for t in pinned))
    hout = torch.empty(progs.P * 3, dtype=torch.float64).pin_memory()
    hout_np = hout.numpy().view(beagle.FITNESS_DTYPE)
    beagle.score_host(hp, ds, out=hout_np, stream=stream)
    e2e_s = []
    for _ in range(args.e2e_steps):
        t0 = time.perf_counter()
        beagle.score_host(hp, ds, out=hout_np, stream=stream)
        e2e_s.append(time.perf_counter() - t0)
    h2d = hp.ops.nbytes + hp.offsets.nbytes + hp.lengths.nbytes + hp.consts.nbytes
    d2h = progs.P * beagle.FITNESS_DTYPE.itemsize

    rates = beagle.measure_op_rates(1.0, stream=stream)
    t_straight = roofline_peak(progs, pr.N, rates)
    kern_avg_s = kern_ms / max(kern_launches, 1) / 1e3
    achieved = node_evals / kern_avg_s / 1e9
    issue = issue_roofline([(progs, pr.N)], clk["sm_mhz"] or 2070.0)
    peak_straight = node_evals / t_straight / 1e9
    peak = node_evals / issue["seconds"] / 1e9 if issue else peak_straight

    if rank != 0:
        return 0
    cpu = cpu_baseline(pr, args.cpu_seconds)
    srt = sorted(step_ms)
    line = {
        "metric": METRIC,
        "value": whole_job_gpops(node_evals, args.steps, world, tot_ms),
        "unit": "GPoPs",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": warm,
        "ms_per_step": tot_ms / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "P": progs.P, "N": pr.N, "d": pr.d,
                   "tokens": progs.tokens, "node_evals_per_step": node_evals,
                   "precision": "fp32-compensated",
                   "l2": "flushed before every timed step (256 MiB write, outside events)",
                   "parallelism": f"replicas x{world} (independent populations)"},
        "p50_ms": srt[len(srt) // 2],
        "p99_ms": srt[min(len(srt) - 1, int(round(0.99 * (len(srt) - 1))))],
        "fp64": {"value": node_evals / (statistics.median(f64_ms) / 1e3) / 1e9,
                 "unit": "GPoPs", "ms_per_step": statistics.median(f64_ms)},
        "fp32c_vs_fp64_speedup": statistics.median(f64_ms) / statistics.median(step_ms),
        "fp32c_error_vs_fp64_path": {
            "programs_compared": int(ok.sum()),
            "frac_within_1e-5": float(within.mean()) if ok.any() else None,
            "median_rel": float(np.median(rel)) if ok.any() else None,
            "note": "fp32 against fp64 evaluation of the programs themselves: ill-conditioned "
                    "random programs differ in their per-case values, not in the aggregation"},
        "fp32c_aggregation_error": agg,
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "GPoPs",
                     "frac": achieved / peak, "traffic": captured_traffic(),
                     "traffic_unit": "bytes per launch (ncu dram read + write)",
                     "peak_basis": ("issue roofline: the op mix's instructions (ncu counts of "
                                    "each operator as implemented, validity check included, "
                                    "leaves free) at 4 issues / SM / cycle, 152 SMs, the "
                                    "measured SM clock; binding: " + issue["binding"])
                                   if issue else "straight-line per-op throughput",
                     "per_pipe_ms": issue["per_pipe_ms"] if issue else None,
                     "peak_straight_line_ops": peak_straight,
                     "frac_straight_line_ops": achieved / peak_straight,
                     "kernel_ms": kern_avg_s * 1e3},
        "cpu_baseline": cpu,
        "e2e": {"value": node_evals / statistics.median(e2e_s) / 1e9, "unit": "GPoPs",
                "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)},
        "gpu_launches": LAUNCHES_PER_CALL * args.steps,
        "clocks": clk,
        "op_rates_gevals": {str(k): v / 1e9 for k, v in sorted(rates.items())},
    }
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
