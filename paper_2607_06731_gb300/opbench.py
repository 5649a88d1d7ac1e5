"""Per-operator throughput of the scoring kernel on single-operator program chains.

    python -m paper_2607_06731_gb300.opbench [--kind ADDX,SIN,...] [--P 20000] [--reps 5]
    python -m paper_2607_06731_gb300.opbench --dispatch

Each population holds P copies of one chain (e.g. ``x0 x1 ADD x2 ADD ...`` for ADDX, the
fused leaf-then-add handler; ``x0 SIN SIN ...`` for SIN) on N = 1024 cases, d = 5. Prints
node evaluations per second next to the straight-line throughput of the same operator
(beagle_measure_op_rates), which shows how much of each operator's cost is interpreter
overhead.
"""
from __future__ import annotations

import argparse
import json

import numpy as np

from . import beagle, synth as S

KINDS = ["ADDX", "MULC", "PDIVX", "PUSH_ADD", "PUSH_MUL", "SQUARE", "PSQRT", "EXP", "PLOG",
         "SIN", "COS"]
ROOF_OP = {"ADDX": S.ADD, "MULC": S.MUL, "PDIVX": S.PDIV, "PUSH_ADD": S.ADD,
           "PUSH_MUL": S.MUL, "SQUARE": S.SQUARE, "PSQRT": S.PSQRT, "EXP": S.EXP,
           "PLOG": S.PLOG, "SIN": S.SIN, "COS": S.COS}


def chain(kind: str, d: int = 5, length: int = 101):
    if kind in ("SIN", "COS", "EXP", "PLOG", "PSQRT", "SQUARE"):
        return [(S.LOAD0, 0.0)] + [(getattr(S, kind), 0.0)] * (length - 1)
    half = (length - 1) // 2
    if kind == "ADDX":
        return [(S.LOAD0, 0.0)] + sum([[(S.LOAD0 + i % d, 0.0), (S.ADD, 0.0)]
                                       for i in range(half)], [])
    if kind == "MULC":
        return [(S.LOAD0, 0.0)] + sum([[(S.CONST, 1.0001), (S.MUL, 0.0)]
                                       for _ in range(half)], [])
    if kind == "PDIVX":
        return [(S.LOAD0, 0.0)] + sum([[(S.LOAD0 + i % d, 0.0), (S.PDIV, 0.0)]
                                       for i in range(half)], [])
    op = S.ADD if kind == "PUSH_ADD" else S.MUL
    toks = []
    for r in range(10):
        toks += [(S.LOAD0 + i % d, 0.0) for i in range(10)] + [(op, 0.0)] * 9
        if r:
            toks.append((op, 0.0))
    return toks


def run(kinds, P=20000, reps=5, N=1024, d=5):
    import torch
    rng = np.random.default_rng(0)
    X = rng.uniform(0.5, 1.5, size=(d, N)).astype(np.float32)
    y = (X[0] + rng.normal(0, 0.1, N)).astype(np.float32)
    ds = beagle.Dataset(X, y)
    rates = beagle.measure_op_rates(1.0)
    out_rows = []
    for kind in kinds:
        prog = chain(kind, d)
        progs = S.from_token_lists([prog] * P)
        dp = beagle.DevicePrograms(progs)
        out = torch.empty((dp.P, 3), dtype=torch.float64, device="cuda")
        for _ in range(2):
            beagle.score_programs(dp, ds, out=out)
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(reps):
            beagle.score_programs(dp, ds, out=out)
        b.record()
        torch.cuda.synchronize()
        ms = a.elapsed_time(b) / reps
        ops = sum(1 for t in prog if t[0] == ROOF_OP[kind])
        row = {"kind": kind, "tokens": len(prog), "ms": round(ms, 4),
               "gpops": round(len(prog) * N * P / ms / 1e6, 1),
               "op_evals_per_s_T": round(ops * N * P / ms / 1e9, 3),
               "straight_line_T": round(rates[ROOF_OP[kind]] / 1e12, 3)}
        row["frac_of_straight_line"] = round(row["op_evals_per_s_T"] / row["straight_line_T"], 3)
        out_rows.append(row)
        print(json.dumps(row), flush=True)
    ds.release()
    return out_rows


def dispatch(warps=(1, 4, 8, 16, 24, 32)):
    """Cost of the bare token dispatch (beagle_measure_dispatch) at several warps per SM."""
    rows = []
    for w in warps:
        c, r = beagle.measure_dispatch(w)
        row = {"warps_per_sm": w, "cycles_per_dispatch": round(c, 1),
               "dispatches_per_sm_cycle": round(r, 4)}
        rows.append(row)
        print(json.dumps(row), flush=True)
    return rows


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--kind", default=",".join(KINDS))
    ap.add_argument("--P", type=int, default=20000)
    ap.add_argument("--reps", type=int, default=5)
    ap.add_argument("--dispatch", action="store_true",
                    help="measure the bare token dispatch instead")
    a = ap.parse_args()
    from . import build
    build.build()
    if a.dispatch:
        dispatch()
    else:
        run(a.kind.split(","), a.P, a.reps)


if __name__ == "__main__":
    main()
