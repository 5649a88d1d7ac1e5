"""Comparison gates between the CUDA path and the oracle.

Random programs can be ill-conditioned (cancellation, exp chains, sin of huge arguments), so
fp32 program arithmetic cannot match an fp64 evaluation within 1e-5 for every program. The
gates therefore run the oracle twice, in FP64 and in FP32-ops mode (every op rounded to
fp32), and call a program *robust* when
  * both oracle runs agree on all flags and neither saw a value within 1e-5 of a threshold
    (oracle NEAR bit),
  * their fitnesses agree within 1e-6, and
  * a first-order bound of the fitness change caused by the per-case output differences
    delta_i = |f32_i - f64_i|, summed without cancellation, is below 1e-6 (relative):
      SSE: 2 sum |e_i| delta_i;   r^2: r^2 (2 sum delta_i |yc_i| / |S_fy| + 2 sum |fc_i| delta_i / S_ff).
    The GPU's fp32 transcendentals differ from the oracle's by a few ulp per op, so a program
    whose outputs move less than 1e-6 under fp32 rounding moves well under 1e-5 on the GPU.
  Gate A  GPU FP32  vs oracle FP32-ops  on robust programs, 1e-5 rel (1e-7 abs)
  Gate B  GPU FP32  vs oracle FP64      on robust programs, 1e-5 rel (1e-7 abs)
  Gate C  GPU FP64  vs oracle FP64      on robust programs, 1e-12 rel (1e-13 abs)
Flags (INVALID, DEGENERATE, MALFORMED) must be equal on robust programs; off the robust set
their mismatches are counted and bounded.
"""
from __future__ import annotations

import numpy as np

import oracle

FLAG_BITS = 1 | 2 | 4
TOL32 = (1e-5, 1e-7)
TOL64 = (1e-12, 1e-13)


def close(a, b, rel, abs_):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    both_inf = np.isinf(a) & np.isinf(b) & (np.sign(a) == np.sign(b))
    with np.errstate(invalid="ignore"):
        ok = np.abs(a - b) <= np.maximum(rel * np.abs(b), abs_)
    return ok | both_inf


def _case_bound_ok(progs, X, y, p, rel):
    ops, cs = progs.program(p)
    f32, fl32 = oracle.eval_program(ops, cs, X, "fp32")
    f64, fl64 = oracle.eval_program(ops, cs, X, "fp64")
    if (fl32 | fl64) & (oracle.F_INVALID | oracle.F_MALFORMED):
        return True                     # decided by the flags alone
    yd = np.asarray(y, np.float64)
    n = len(yd)
    dlt = np.abs(f32 - f64)
    e = f64 - yd
    sse = float(e @ e)
    if 2.0 * float(np.abs(e) @ dlt) > max(rel * sse, 1e-8 * n):
        return False
    yc = yd - yd.mean()
    syy = float(yc @ yc)
    fc = f64 - f64.mean()
    sff = float(fc @ fc)
    sfy = float(fc @ yc)
    if sff == 0.0 or sfy == 0.0:
        return True
    r2 = sfy * sfy / (sff * syy)
    br = r2 * (2.0 * float(dlt @ np.abs(yc)) / abs(sfy) + 2.0 * float(np.abs(fc) @ dlt) / sff)
    return br <= max(rel * abs(1.0 - r2), 1e-8)


def robust_set(o32, o64, progs=None, X=None, y=None, rel=1e-6):
    m32, r32, f32 = o32
    m64, r64, f64 = o64
    same_flags = (f32 & FLAG_BITS) == (f64 & FLAG_BITS)
    near = ((f32 | f64) & oracle.F_NEAR) != 0
    rob = same_flags & ~near & close(m32, m64, rel, 1e-9) & close(r32, r64, rel, 1e-9)
    if progs is not None:
        from concurrent.futures import ThreadPoolExecutor
        idx = np.nonzero(rob)[0]
        with ThreadPoolExecutor(max(1, oracle.threads())) as ex:
            ok = list(ex.map(lambda p: _case_bound_ok(progs, X, y, int(p), rel), idx))
        rob[idx[~np.asarray(ok, bool)]] = False
    return rob


def gate(gpu, ref, mask, tol):
    gm, gr, gf = gpu
    om, orr, of = ref
    flags_ok = (gf & FLAG_BITS) == (of & FLAG_BITS)
    val_ok = close(gm, om, *tol) & close(gr, orr, *tol)
    bad = mask & ~(flags_ok & val_ok)
    return np.nonzero(bad)[0]


def describe(idx, gpu, ref, limit=5):
    gm, gr, gf = gpu
    om, orr, of = ref
    lines = []
    for i in idx[:limit]:
        lines.append(f"p={i} gpu=({gm[i]:.9g}, {gr[i]:.9g}, {gf[i]}) "
                     f"oracle=({om[i]:.9g}, {orr[i]:.9g}, {of[i]})")
    return "\n".join(lines)


def check_fp32(gpu, o32, o64, rob, min_robust=0.4, max_flag_mismatch=0.005):
    """Gates A and B plus the flag rule on the robust set rob; returns its fraction."""
    frac = float(rob.mean()) if len(rob) else 1.0
    assert frac >= min_robust, f"robust fraction {frac:.3f} < {min_robust}"
    a = gate(gpu, o32, rob, TOL32)
    assert len(a) == 0, "gate A (vs FP32-ops oracle):\n" + describe(a, gpu, o32)
    b = gate(gpu, o64, rob, TOL32)
    assert len(b) == 0, "gate B (vs FP64 oracle):\n" + describe(b, gpu, o64)
    nonnear = (o32[2] & oracle.F_NEAR) == 0
    mism = nonnear & ((gpu[2] & FLAG_BITS) != (o32[2] & FLAG_BITS))
    assert mism.mean() <= max_flag_mismatch, (
        f"flag mismatch on {int(mism.sum())} non-NEAR programs:\n"
        + describe(np.nonzero(mism)[0], gpu, o32))
    return frac


def check_fp64(gpu, o32, o64, rob):
    c = gate(gpu, o64, rob, TOL64)
    assert len(c) == 0, "gate C (FP64 path vs FP64 oracle):\n" + describe(c, gpu, o64)
    nonnear = (o64[2] & oracle.F_NEAR) == 0
    mism = nonnear & ((gpu[2] & FLAG_BITS) != (o64[2] & FLAG_BITS))
    assert mism.mean() <= 0.005, describe(np.nonzero(mism)[0], gpu, o64)
