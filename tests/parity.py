"""Comparison gates between the CUDA path and the oracle.

Random programs can be ill-conditioned (cancellation, exp chains, sin of huge arguments), so
fp32 program arithmetic cannot match an fp64 evaluation within 1e-5 for every program. The
gates therefore use the oracle twice, in FP64 and in FP32-ops mode (every op rounded to
fp32), and call a program *robust* when both oracle runs agree within 1e-6 and on all flags,
and neither saw a value within 1e-5 of a threshold (oracle NEAR bit):
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


def robust_set(o32, o64):
    m32, r32, f32 = o32
    m64, r64, f64 = o64
    same_flags = (f32 & FLAG_BITS) == (f64 & FLAG_BITS)
    near = ((f32 | f64) & oracle.F_NEAR) != 0
    return (same_flags & ~near & close(m32, m64, 1e-6, 1e-9) & close(r32, r64, 1e-6, 1e-9))


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


def check_fp32(gpu, o32, o64, min_robust=0.8, max_flag_mismatch=0.005):
    """Gates A and B plus the flag rule; returns the robust fraction."""
    rob = robust_set(o32, o64)
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


def check_fp64(gpu, o32, o64):
    rob = robust_set(o32, o64)
    c = gate(gpu, o64, rob, TOL64)
    assert len(c) == 0, "gate C (FP64 path vs FP64 oracle):\n" + describe(c, gpu, o64)
    nonnear = (o64[2] & oracle.F_NEAR) == 0
    mism = nonnear & ((gpu[2] & FLAG_BITS) != (o64[2] & FLAG_BITS))
    assert mism.mean() <= 0.005, describe(np.nonzero(mism)[0], gpu, o64)
