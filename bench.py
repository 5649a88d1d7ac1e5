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
WORKLOAD = ("c2-population-100k: P=100000 programs, length U{16..128}, d=5, N=1024 cases, "
            "X~U[-3,3], y=20-node expression + N(0,0.01) noise; MSE and 1-R^2")


def parse():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--fp64-steps", type=int, default=3)
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--P", type=int, default=100_000)
    ap.add_argument("--cpu-seconds", type=float, default=10.0,
                    help="target wall time of the CPU oracle sample")
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
    n = 200
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
    return {"value": evals / dt / 1e9, "unit": "GPoPs", "cores": oracle.threads(),
            "kind": "oracle",
            "sample": f"{n2} of {pr.programs.P} programs (seeded) x all {pr.N} cases, FP64 "
                      f"oracle, {dt:.1f} s wall"}


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


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.impl == "reference":
        return run_reference(args, rank, world)

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

    for _ in range(max(3, args.warmup)):
        flush.zero_()
        step()
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
    if dist is not None:
        t = torch.tensor([tot_ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        tot_ms = float(t.item())
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
    t_roof = roofline_peak(progs, pr.N, rates)
    kern_avg_s = kern_ms / max(kern_launches, 1) / 1e3
    achieved = node_evals / kern_avg_s / 1e9
    peak = node_evals / t_roof / 1e9

    if rank != 0:
        return 0
    cpu = cpu_baseline(pr, args.cpu_seconds)
    srt = sorted(step_ms)
    line = {
        "metric": METRIC,
        "value": node_evals * args.steps * world / (tot_ms / 1e3) / 1e9,
        "unit": "GPoPs",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": max(3, args.warmup),
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
            "median_rel": float(np.median(rel)) if ok.any() else None},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "GPoPs",
                     "frac": achieved / peak, "traffic": None,
                     "peak_basis": "per-op throughput measured by beagle_measure_op_rates "
                                   "on this GPU (validity check included, leaves free)",
                     "kernel_ms": kern_avg_s * 1e3},
        "cpu_baseline": cpu,
        "e2e": {"value": node_evals / statistics.median(e2e_s) / 1e9, "unit": "GPoPs",
                "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)},
        "gpu_launches": 2 * args.steps,
        "clocks": clk,
        "op_rates_gevals": {str(k): v / 1e9 for k, v in sorted(rates.items())},
    }
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
