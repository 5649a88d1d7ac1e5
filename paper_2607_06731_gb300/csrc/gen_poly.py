"""Derive the constants of the FP32 path's sin, cos and log (transcend.cuh).

    python paper_2607_06731_gb300/csrc/gen_poly.py

Prints, as fp32 hex literals:
  * pi/2 split into three fp32 parts (C1 + C2 + C3, each the fp32 rounding of what the
    previous parts leave), and 2/pi, for Cody and Waite's additive range reduction;
  * near-minimax polynomials on |r| <= (pi/4)(1.01) (1 % margin for a quotient rounded off
    by one), in s = r^2: sin r = r + r^3 P(s) and cos r = 1 + s Q(s), P and Q of degree 3,
    fitted to relative error by weighted least squares on Chebyshev nodes with Lawson
    reweighting, then rounded to fp32; the script reports the resulting maximum relative
    error with exact evaluation;
  * ln 2 in two fp32 parts and ln(1 + f) = f + f^2 (-1/2 + f L(f)) with L of degree 7 on f in [sqrt(1/2) - 1,
    sqrt(2) - 1] (the mantissa m of the argument taken into [sqrt(1/2), sqrt(2))).
"""
import mpmath as mp
import numpy as np

mp.mp.dps = 60


def f32(x):
    return np.float32(float(x))


def hexf(x):
    m, e = float(np.float32(x)).hex().split("p")
    m = m.rstrip("0")
    return (m + "0" if m.endswith(".") else m) + "p" + e + "f"


def fit(target, weight, b, deg, npts=300, iters=40, a=0):
    nodes = [(a + b) / 2 + (b - a) / 2 * mp.cos(mp.pi * (2 * k + 1) / (2 * npts))
             for k in range(npts)]
    w = [weight(x) for x in nodes]
    for _ in range(iters):
        A = mp.matrix(npts, deg + 1)
        rhs = mp.matrix(npts, 1)
        for i, x in enumerate(nodes):
            for j in range(deg + 1):
                A[i, j] = w[i] * x ** j
            rhs[i] = w[i] * target(x)
        c = mp.lu_solve(A.T * A, A.T * rhs)
        err = [abs(sum(c[j] * x ** j for j in range(deg + 1)) - target(x)) * weight(x)
               for x in nodes]
        m = max(err)
        w = [w[i] * (1 + (err[i] / m) ** 2) for i in range(npts)]
    return [c[j] for j in range(deg + 1)]


def max_rel(fn, ref, b, n=20001, a=1e-6):
    worst = mp.mpf(0)
    for x in np.linspace(float(a), float(b), n):
        x = mp.mpf(x)
        if x == 0:
            continue
        worst = max(worst, abs(fn(x) - ref(x)) / abs(ref(x)))
    return worst


def main():
    half_pi = mp.pi / 2
    c1 = f32(half_pi)
    c2 = f32(half_pi - mp.mpf(float(c1)))
    c3 = f32(half_pi - mp.mpf(float(c1)) - mp.mpf(float(c2)))
    print("two_over_pi", hexf(f32(2 / mp.pi)))
    print("pio2 parts", hexf(c1), hexf(c2), hexf(c3))
    b = (mp.pi / 4 * mp.mpf("1.01")) ** 2
    P = fit(lambda s: (mp.sin(mp.sqrt(s)) - mp.sqrt(s)) / s ** 1.5 if s > 0 else mp.mpf(-1) / 6,
            lambda s: s ** 1.5 / mp.sin(mp.sqrt(s)) if s > 0 else mp.mpf(0), b, 3)
    Q = fit(lambda s: (mp.cos(mp.sqrt(s)) - 1) / s if s > 0 else mp.mpf(-1) / 2,
            lambda s: s / mp.cos(mp.sqrt(s)), b, 3)
    P32 = [f32(v) for v in P]
    Q32 = [f32(v) for v in Q]

    def horner(c, s):
        v = mp.mpf(0)
        for x in reversed(c):
            v = v * s + mp.mpf(float(x))
        return v
    es = max_rel(lambda r: r + r ** 3 * horner(P32, r * r), mp.sin, mp.sqrt(b))
    ec = max_rel(lambda r: 1 + r * r * horner(Q32, r * r), mp.cos, mp.sqrt(b))
    print("sin P", " ".join(hexf(v) for v in P32), "max rel err %.3e" % es)
    print("cos Q", " ".join(hexf(v) for v in Q32), "max rel err %.3e" % ec)

    ln2 = mp.log(2)
    h = f32(ln2)
    ln2 = mp.log(2)
    h = f32(ln2)
    print("ln2 parts", hexf(h), hexf(f32(ln2 - mp.mpf(float(h)))))
    lo, hi = mp.sqrt(mp.mpf(1) / 2) - 1, mp.sqrt(2) - 1
    Lc = fit(lambda f: (mp.log(1 + f) - f + f * f / 2) / f ** 3 if f != 0 else mp.mpf(1) / 3,
             lambda f: abs(f ** 3 / mp.log(1 + f)) if f != 0 else mp.mpf(0), hi, 7, a=lo)
    L32 = [f32(v) for v in Lc]
    el = max_rel(lambda f: f + f * f * (mp.mpf(-0.5) + f * horner(L32, f)),
                 lambda f: mp.log(1 + f), hi, a=lo)
    print("log L", " ".join(hexf(v) for v in L32), "max rel err %.3e" % el)


if __name__ == "__main__":
    main()
