"""Parity of the CUDA scoring path (through the C ABI) with the oracle, on the GPU."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_2607_06731_gb300 import beagle, synth as S
from tests import parity
from tests.gcl_text import paper_genomes

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    yield


def run_gpu(progs, X, y, precision="fp32c", ds=None):
    own = ds is None
    if own:
        ds = beagle.Dataset(X, y)
    dp = beagle.DevicePrograms(progs)
    out = beagle.score_programs(dp, ds, precision=precision)
    torch.cuda.synchronize()
    r = beagle.unpack_fitness(out)
    if own:
        ds.release()
    return r


def full_check(progs, X, y, min_strict=0.0, fp64=True, name=None):
    refs = parity.references(progs, X, y)
    g32 = run_gpu(progs, X, y, "fp32c")
    stats = parity.check_fp32(g32, refs, min_strict=min_strict, name=name)
    if fp64:
        g64 = run_gpu(progs, X, y, "fp64")
        stats["fp64"] = parity.check_fp64(g64, refs, name=name)
    return stats


def test_c1_plain_scoring_full_size():
    """P = 1024 programs of length 8-32 on N = 1024 cases, d = 2 (one tile)."""
    pr = S.make_c1()
    stats = full_check(pr.programs, pr.X, pr.y, min_strict=0.3, name="c1")
    print(f"c1 {stats}")


def test_c2_distribution_small_population():
    pr = S.make_c2(P=3000)
    full_check(pr.programs, pr.X, pr.y, name="c2-3000")


@pytest.mark.parametrize("N,d", [(2500, 10), (700, 16), (2, 1), (1025, 3), (3000, 13),
                                 (1024, 12), (4096, 5)])
def test_multi_tile_and_ragged_tail(N, d):
    rng = np.random.default_rng(N * 31 + d)
    X = rng.uniform(-3, 3, size=(d, N)).astype(np.float32)
    y = (np.sin(X[0]) * 2 + X[-1] + rng.normal(0, 0.1, N)).astype(np.float32)
    progs = S.gen_programs(rng, 500, 4, 64, d)
    full_check(progs, X, y, name=f"tiles-{N}-{d}")


def test_c2_full_population_sampled():
    """The bench workload (P = 100,000, L 16-128, d = 5, N = 1024) in the launch bench.py
    times; a seeded sample of programs is checked against the oracle one by one."""
    pr = S.make_c2()
    g32 = run_gpu(pr.programs, pr.X, pr.y, "fp32c")
    idx = np.random.default_rng(0).choice(pr.programs.P, 1500, replace=False)
    sub = pr.programs.subset(idx)
    refs = parity.references(sub, pr.X, pr.y)
    print(parity.check_fp32(tuple(a[idx] for a in g32), refs, name="c2-full-1500"))


def test_c3_full_size_sampled():
    """P = 50,000 programs on N = 1,000,000 cases (977 tiles): every program scored on the
    GPU, a seeded 500-program sample checked against the oracle (with its error bound) at the
    full case count. The FP64 path is checked on the sample."""
    pr = S.make_c3()
    ds = beagle.Dataset(pr.X, pr.y)
    g32 = run_gpu(pr.programs, pr.X, pr.y, "fp32c", ds=ds)
    idx = np.random.default_rng(1).choice(pr.programs.P, 500, replace=False)
    sub = pr.programs.subset(idx)
    refs = parity.references(sub, pr.X, pr.y)
    print(parity.check_fp32(tuple(a[idx] for a in g32), refs, name="c3-500"))
    g64 = run_gpu(sub, pr.X, pr.y, "fp64", ds=ds)
    parity.check_fp64(g64, refs, name="c3-500")
    ds.release()


def _quadratic(n=1024, seed=3):
    rng = np.random.default_rng(seed)
    a = rng.uniform(0.2, 3.0, n) * rng.choice([-1, 1], n)
    b = rng.uniform(-6, 6, n)
    c = rng.uniform(-3, 3, n)
    X = np.stack([a, b, c]).astype(np.float32)
    A, B, C = (X[i].astype(np.float64) for i in range(3))
    X = X[:, B * B - 4 * A * C >= 0]
    A, B, C = (X[i].astype(np.float64) for i in range(3))
    y = ((-B + np.sqrt(B * B - 4 * A * C)) / (2 * A)).astype(np.float32)
    return X, y


def test_paper_genomes_on_gpu():
    """"Understanding Beagle Output"'s genomes (DUP, DEL, DIV by self, SQUARE) solve the quadratic."""
    X, y = _quadratic()
    progs = S.from_token_lists([t for _, t in paper_genomes().values()])
    refs = parity.references(progs, X, y)
    g32 = run_gpu(progs, X, y, "fp32c")
    g64 = run_gpu(progs, X, y, "fp64")
    parity.check_fp32(g32, refs)
    parity.check_fp64(g64, refs)
    assert np.all(g64[1] < 1e-12) and np.all(g32[1] < 1e-6)
    assert np.all(g32[2] == 0)


def _stack_ops_programs(rng, P, d):
    """Random programs that also use DUP, SWAP and DEL."""
    progs = []
    for _ in range(P):
        L = int(rng.integers(3, 40))
        toks, depth = [], 0
        for t in range(L):
            r = L - t
            choices = []
            if depth + 1 <= 16 and depth <= r - 1:
                choices += ["leaf", "leaf", "dup"] if depth >= 1 else ["leaf"]
            if depth >= 1 and depth - 1 <= r - 1:
                choices += ["un"]
            if depth >= 2 and depth - 2 <= r - 1:
                choices += ["bin", "bin", "del"]
            if depth >= 1 and depth - 1 <= r - 1 and depth >= 2:
                choices += ["swap"]
            k = choices[int(rng.integers(len(choices)))]
            if k == "dup" and depth + 1 > 16:
                k = "un"
            if k == "leaf":
                if rng.random() < 0.5:
                    toks.append((S.LOAD0 + int(rng.integers(d)), 0.0))
                else:
                    toks.append((S.CONST, float(np.float32(rng.uniform(-2, 2)))))
                depth += 1
            elif k == "dup":
                toks.append((S.DUP, 0.0)); depth += 1
            elif k == "un":
                toks.append((int(rng.choice(S.UNARY)), 0.0))
            elif k == "swap":
                toks.append((S.SWAP, 0.0))
            elif k == "del":
                toks.append((S.DEL, 0.0)); depth -= 1
            else:
                toks.append((int(rng.choice(S.BINARY)), 0.0)); depth -= 1
        if depth == 1 and oracle.check_program([t[0] for t in toks], d, 16) == 0:
            progs.append(toks)
    return S.from_token_lists(progs)


def test_dup_swap_del():
    rng = np.random.default_rng(17)
    d = 3
    progs = _stack_ops_programs(rng, 800, d)
    assert progs.P > 300
    X = rng.uniform(-3, 3, size=(d, 1500)).astype(np.float32)
    y = (X[0] * X[1] + rng.normal(0, 0.1, 1500)).astype(np.float32)
    full_check(progs, X, y)


def test_malformed_programs_are_flagged():
    C, L0 = S.CONST, S.LOAD0
    good = [(C, 1.5), (L0, 0), (S.ADD, 0)]
    bad = [
        [(S.ADD, 0)],                                   # underflow
        [(C, 1.0), (C, 2.0)],                           # two values left
        [(L0 + 3, 0)],                                  # x3 with d = 2
        [(99, 0)],                                      # unknown opcode
        [(C, 1.0)] * 33 + [(S.ADD, 0)] * 32,            # 33 values > BEAGLE_MAX_DEPTH
        [(C, 1.0)] + [(S.SIN, 0)] * 256,                # 257 tokens > BEAGLE_MAX_LENGTH
        [(L0, 0), (S.COPY0, 0)] + [(C, 1.0)] * 31 + [(S.ADD, 0)] * 31 +
        [(S.PASTE0, 0), (S.ADD, 0)],                    # 32 values + a live variable
    ]
    ok_deep = [(C, 1.0)] * 32 + [(S.ADD, 0)] * 31       # exactly 32 deep (the deep pass)
    ok_long = [(L0, 0)] + [(S.SIN, 0)] * 255            # exactly 256 tokens
    progs = S.from_token_lists([good] + bad + [ok_deep, ok_long])
    X = np.random.default_rng(0).uniform(-1, 1, size=(2, 300)).astype(np.float32)
    y = X[0].copy()
    for prec in ("fp32c", "fp64"):
        m, r, f = run_gpu(progs, X, y, prec)
        assert f[0] == 0
        assert np.all(f[1:1 + len(bad)] == beagle.FLAG_MALFORMED), f
        assert np.all(np.isinf(m[1:1 + len(bad)]))
        assert f[-2] & beagle.FLAG_MALFORMED == 0 and f[-1] & beagle.FLAG_MALFORMED == 0
    okp = S.from_token_lists([good, ok_deep, ok_long])
    g32 = run_gpu(okp, X, y, "fp32c")
    parity.check_fp32(g32, parity.references(okp, X, y))


def _deep_population(rng, P, d):
    """Programs of every depth up to the paper's StackSize of 32, shallow and deep mixed (and
    some with COPY/PASTE variables)."""
    progs = S.gen_programs(rng, P, 30, 200, d, depth_cap=32, weights=(0.55, 0.1, 0.35),
                           unary=S.ALL_UNARY, binary=S.ALL_BINARY)
    depth = np.array([S.max_depth(progs.program(p)[0]) for p in range(progs.P)])
    return progs, depth


@pytest.mark.parametrize("cases", [4, 2, 8])
def test_deep_programs_up_to_stack_size_32(cases):
    """Programs deeper than the fast pass's 16-value stack run in the deep pass (32 values):
    parity with the oracle at several tile counts, mixed with shallow programs."""
    rng = np.random.default_rng(40 + cases)
    d, N = 3, 1300
    X = rng.uniform(-1.5, 1.5, (d, N)).astype(np.float32)
    y = (X[0] * X[1] - np.tanh(X[2])).astype(np.float32)
    progs, depth = _deep_population(rng, 500, d)
    assert (depth > 16).sum() >= 100 and (depth <= 16).sum() >= 50 and depth.max() <= 32
    refs = parity.references(progs, X, y)
    beagle.set_launch_config(cases_per_lane=cases)
    try:
        g32 = run_gpu(progs, X, y, "fp32c")
        assert not np.any(g32[2] & beagle.FLAG_MALFORMED)
        parity.check_fp32(g32, refs, name=f"deep-{cases}")
        if cases == 4:
            g64 = run_gpu(progs, X, y, "fp64")
            parity.check_fp64(g64, refs, name="deep")
    finally:
        beagle.reset_launch_config()


def test_deep_programs_same_bits_alone_in_batch_and_static():
    rng = np.random.default_rng(44)
    d, N = 2, 900
    X = rng.uniform(-1, 1, (d, N)).astype(np.float32)
    y = (X[0] - X[1] ** 2).astype(np.float32)
    progs, depth = _deep_population(rng, 300, d)
    ds = beagle.Dataset(X, y)
    dp = beagle.DevicePrograms(progs)
    alone = beagle.unpack_fitness(beagle.score_programs(dp, ds))
    out = torch.empty((dp.P, 3), dtype=torch.float64, device="cuda")
    other = S.gen_programs(rng, 700, 4, 60, d)
    dpo = beagle.DevicePrograms(other)
    outo = torch.empty((dpo.P, 3), dtype=torch.float64, device="cuda")
    beagle.score_batch([(dpo, ds, outo), (dp, ds, out)])
    torch.cuda.synchronize()
    for a, b in zip(beagle.unpack_fitness(out), alone):
        assert np.array_equal(a, b, equal_nan=True)
    st = torch.empty((dp.P, 3), dtype=torch.float64, device="cuda")
    beagle.check(beagle.lib().beagle_score_static(
        dp.ops.data_ptr(), dp.offsets.data_ptr(), dp.lengths.data_ptr(), dp.consts.data_ptr(),
        dp.P, ds.id, st.data_ptr(), beagle.FP32_COMPENSATED,
        torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    for a, b in zip(beagle.unpack_fitness(st), alone):
        assert np.array_equal(a, b, equal_nan=True)
    ds.release()


def test_invalid_values_and_constants():
    C = S.CONST
    progs = S.from_token_lists([
        [(C, float("inf"))],                            # non-finite constant
        [(C, 100.0), (S.EXP, 0)],                       # e^100 > 1e30
        [(C, 1.0), (C, 1e16), (C, 1e15), (S.MUL, 0), (S.PDIV, 0)],   # hidden 1e31
        [(C, 2.0 ** 49), (S.SQUARE, 0)],                # 2^98 < 1e30: valid
        [(S.LOAD0, 0), (C, 80.0), (S.MUL, 0), (S.EXP, 0)],   # e^80 > 1e30 on some cases
    ])
    X = np.linspace(-1, 1, 1000, dtype=np.float32).reshape(1, -1)
    y = X[0] * 2
    for prec in ("fp32c", "fp64"):
        m, r, f = run_gpu(progs, X, y, prec)
        assert list(f) == [1, 1, 1, 2, 1], (prec, f)     # 2^98 is valid (and constant)
        assert np.isinf(m[0]) and np.isinf(r[0])


def test_constant_outputs_are_degenerate_across_tiles():
    progs = S.from_token_lists([[(S.CONST, 1.25)],
                                [(S.LOAD0, 0), (S.LOAD0, 0), (S.SUB, 0)],
                                [(S.LOAD0, 0), (S.SIN, 0)]])
    X = np.random.default_rng(2).uniform(-2, 2, size=(1, 3000)).astype(np.float32)
    y = (X[0] ** 2).astype(np.float32)
    for prec in ("fp32c", "fp64"):
        m, r, f = run_gpu(progs, X, y, prec)
        assert list(f) == [2, 2, 0] and r[0] == 1.0 and r[1] == 1.0
        want = np.mean((1.25 - y.astype(np.float64)) ** 2)
        assert abs(m[0] - want) <= 1e-6 * want


def test_outliers_and_large_values_in_tile_statistics():
    """Outputs with a few huge values (at tile starts, inside the first 128 cases, or later),
    offsets far from zero, outputs and targets near 2^52 (unscaled sums) and outputs near 2^70,
    whose squares overflow fp32 (the scaled two-pass sums)."""
    rng = np.random.default_rng(11)
    N = 3000
    X = rng.uniform(-1, 1, size=(3, N)).astype(np.float32)
    X[1, ::512] = 1e4                          # an outlier at every 512-case tile start
    X[1, 256::512] = -3e3                      # ... and at the other 256-case tile starts
    X[2, rng.integers(0, N, 12)] = 5e5         # scattered outliers
    X[2, 700:710] = -2e5
    y = (X[0] * 3 + 1).astype(np.float32)
    C, L0, L1, L2 = S.CONST, S.LOAD0, S.LOAD0 + 1, S.LOAD0 + 2
    progs = S.from_token_lists([
        [(L1, 0)],
        [(L1, 0), (S.SQUARE, 0)],
        [(L2, 0), (L0, 0), (S.ADD, 0)],
        [(L2, 0), (C, 1e4), (S.ADD, 0)],                    # offset far from zero
        [(L0, 0), (C, 2.0 ** 52), (S.MUL, 0)],              # outputs near 2^52
        [(L0, 0), (C, 2.0 ** 70), (S.MUL, 0)],              # squares overflow fp32: scaled path
        [(L1, 0), (C, 2.0 ** 40), (S.MUL, 0)],              # above 2^50 at the outliers only
        [(L0, 0), (C, 3.0), (S.MUL, 0), (C, 1.0), (S.ADD, 0)],   # exact fit
    ])
    full_check(progs, X, y)
    yb = (X[0] * 2.0 ** 52).astype(np.float32)           # targets near 2^52
    full_check(progs, X, yb)


def test_empty_population():
    X = np.ones((1, 4), np.float32) * np.arange(4, dtype=np.float32)
    ds = beagle.Dataset(X, X[0])
    e = torch.empty(0, dtype=torch.uint8, device="cuda")
    out = beagle.score(e, e.long(), e.int(), e.float(), ds)
    torch.cuda.synchronize()
    assert out.shape == (0, 3)
    ds.release()


def test_same_bits_alone_and_in_a_mix():
    """Fixed-order reductions: a program's fitness does not depend on its neighbours."""
    pr = S.make_c2(P=4000, N=3000)
    ds = beagle.Dataset(pr.X, pr.y)
    full = run_gpu(pr.programs, pr.X, pr.y, "fp32c", ds=ds)
    idx = np.random.default_rng(4).choice(pr.programs.P, 300, replace=False)
    alone = run_gpu(pr.programs.subset(idx), pr.X, pr.y, "fp32c", ds=ds)
    for a, b in zip(full, alone):
        assert np.array_equal(a[idx], b, equal_nan=True)
    again = run_gpu(pr.programs, pr.X, pr.y, "fp32c", ds=ds)
    for a, b in zip(full, again):
        assert np.array_equal(a, b, equal_nan=True)
    ds.release()


def test_score_host_matches_device_call():
    pr = S.make_c1(P=500)
    ds = beagle.Dataset(pr.X, pr.y)
    dev = run_gpu(pr.programs, pr.X, pr.y, "fp32c", ds=ds)
    host = beagle.unpack_fitness(beagle.score_host(pr.programs, ds, precision="fp32c"))
    for a, b in zip(dev, host):
        assert np.array_equal(a, b, equal_nan=True)
    ds.release()


def test_dataset_upload_from_device_and_rejections():
    rng = np.random.default_rng(0)
    X = rng.uniform(-1, 1, size=(3, 100)).astype(np.float32)
    y = X[0] + X[1]
    a = beagle.Dataset(X, y)
    b = beagle.Dataset(torch.from_numpy(X).cuda(), torch.from_numpy(y).cuda())
    assert abs(a.ybar - b.ybar) == 0 and a.syy == b.syy
    pr = S.gen_programs(rng, 50, 4, 20, 3)
    ra = run_gpu(pr, X, y, ds=a)
    rb = run_gpu(pr, X, y, ds=b)
    assert np.array_equal(ra[0], rb[0], equal_nan=True)
    a.release(), b.release()
    with pytest.raises(beagle.BeagleError):
        beagle.Dataset(X, np.ones(100, np.float32))          # constant y
    Xn = X.copy(); Xn[1, 5] = np.nan
    with pytest.raises(beagle.BeagleError):
        beagle.Dataset(Xn, y)
    with pytest.raises(beagle.BeagleError):
        beagle.Dataset(np.ones((17, 10), np.float32), np.arange(10, dtype=np.float32))


def _eval_gpu(progs, X, y, precision):
    ds = beagle.Dataset(X, y)
    dp = beagle.DevicePrograms(progs)
    outs, fit = beagle.eval_programs(dp, ds, precision=precision)
    torch.cuda.synchronize()
    r = outs.cpu().numpy(), beagle.unpack_fitness(fit)
    ds.release()
    return r


@pytest.mark.parametrize("N,d", [(1024, 5), (1500, 3), (700, 16)])
def test_ieee_ops_bit_exact_per_case(N, d):
    """With only + - * pdiv psqrt square, every op is correctly rounded in both precisions,
    so the per-case outputs (beagle_eval) must equal the oracle's bit for bit."""
    rng = np.random.default_rng(N + d)
    X = rng.uniform(-3, 3, size=(d, N)).astype(np.float32)
    y = (X[0] * X[-1]).astype(np.float32)
    progs = S.gen_programs(rng, 400, 4, 96, d, unary=(S.SQUARE, S.PSQRT), binary=S.BINARY)
    for prec, mode in (("fp32c", "fp32"), ("fp64", "fp64")):
        outs, (m, r, f) = _eval_gpu(progs, X, y, prec)
        for p in range(progs.P):
            ops, cs = progs.program(p)
            fo, fl = oracle.eval_program(ops, cs, X, mode)
            assert (f[p] & 1) == (fl & 1), (prec, p)
            if fl & 1:
                continue
            got = outs[p].astype(np.float64)
            assert np.array_equal(got, fo), (prec, p, np.nonzero(got != fo)[0][:5])


def test_eval_outputs_within_error_bound_per_case():
    """Per-case outputs with transcendentals (beagle_eval): within the oracle's running error
    bound of the FP32-ops value on every case of every non-ambiguous program; FP64 path
    likewise against the FP64 oracle."""
    pr = S.make_c1(P=400, N=1500)
    for prec, mode in (("fp32c", "fp32"), ("fp64", "fp64")):
        outs, _ = _eval_gpu(pr.programs, pr.X, pr.y, prec)
        checked = 0
        for p in range(pr.programs.P):
            ops, cs = pr.programs.program(p)
            f, dl, fl = oracle.eval_bound(ops, cs, pr.X, mode)
            if fl & (oracle.F_INVALID | oracle.F_AMBIG):
                continue
            g = outs[p].astype(np.float64)
            slack = np.spacing(np.abs(f).astype(np.float32 if mode == "fp32" else np.float64))
            bad = np.abs(g - f) > dl + slack
            assert not bad.any(), (prec, p, np.nonzero(bad)[0][:5], g[bad][:3], f[bad][:3],
                                   dl[bad][:3])
            checked += len(g)
        assert checked > 300000


@pytest.mark.parametrize("cases", [4, 8])
def test_deep_well_conditioned_programs(cases):
    """Deep programs whose values stay well conditioned (positive leaves; +, x and squaring
    only), so that nearly all fall in the strict set: the deep pass (32-value stack) within
    1e-5 of both oracles (1e-12 on the FP64 path), not only inside the error envelope."""
    rng = np.random.default_rng(60 + cases)
    d, N = 3, 1100
    X = rng.uniform(0.5, 1.5, (d, N)).astype(np.float32)
    y = (np.sin(3 * X[0]) + X[1] - X[2]).astype(np.float32)
    progs = S.gen_programs(rng, 400, 56, 100, d, depth_cap=32, weights=(0.68, 0.02, 0.3),
                           unary=(S.SQUARE,), binary=(S.ADD, S.MUL), const_lo=0.5, const_hi=1.5)
    depth = np.array([S.max_depth(progs.program(p)[0]) for p in range(progs.P)])
    assert (depth > 16).sum() >= 200, (depth > 16).sum()
    refs = parity.references(progs, X, y)
    beagle.set_launch_config(cases_per_lane=cases)
    try:
        g32 = run_gpu(progs, X, y, "fp32c")
        assert not np.any(g32[2] & beagle.FLAG_MALFORMED)
        stats = parity.check_fp32(g32, refs, min_strict=0.95, name=f"deep-wc-{cases}")
        print(stats)
        if cases == 4:
            g64 = run_gpu(progs, X, y, "fp64")
            parity.check_fp64(g64, refs, min_strict=0.95, name="deep-wc")
    finally:
        beagle.reset_launch_config()


def _const_heavy_programs(rng, P, d):
    """Programs whose constant subexpressions the packing kernel folds: constants combined by
    every operator kind (transcendentals, protected division and log, DUP, SWAP and DEL on
    constants), mixed with inputs; some fold to invalid values (exp(100), 1e20 * 1e20)."""
    C = S.CONST
    pieces = [
        [(C, 0.7), (S.SIN, 0)], [(C, 1.3), (C, -0.4), (S.PDIV, 0)], [(C, 2.0), (S.PLOG, 0)],
        [(C, 0.3), (S.EXP, 0), (S.COS, 0)], [(C, -2.5), (S.PSQRT, 0), (S.SQUARE, 0)],
        [(C, 0.2), (S.DUP, 0), (S.MUL, 0)], [(C, 1.5), (C, 0.25), (S.SWAP, 0), (S.SUB, 0)],
        [(C, 3.0), (C, 9.0), (S.DEL, 0)], [(C, 0.5), (C, 0.0005), (S.PDIV, 0)],
        [(C, 1.1), (C, 2.2), (S.POW, 0)], [(C, 0.9), (S.TANH, 0), (S.SIGN, 0), (S.CUBE, 0)],
    ]
    bad = [[(C, 100.0), (S.EXP, 0)], [(C, 1e20), (C, 1e20), (S.MUL, 0)]]
    progs = []
    for i in range(P):
        toks = [(S.LOAD0 + int(rng.integers(d)), 0.0)]
        for _ in range(int(rng.integers(1, 6))):
            piece = bad[int(rng.integers(2))] if rng.random() < 0.05 else \
                pieces[int(rng.integers(len(pieces)))]
            toks += piece + [(int(rng.choice([S.ADD, S.SUB, S.MUL, S.PDIV])), 0.0)]
            if rng.random() < 0.4:
                toks += [(S.LOAD0 + int(rng.integers(d)), 0.0), (S.MUL, 0.0)]
        progs.append(toks)
    return S.from_token_lists(progs)


def test_constant_folding_same_bits_and_oracle():
    """Constant subexpressions folded by the packing kernel: every program gives the bits it
    gives when each work item packs it unfolded (programs in the caller's order), on the
    scores and on every case's output, and agrees with the oracle."""
    rng = np.random.default_rng(77)
    d, N = 3, 1300
    X = rng.uniform(-2, 2, (d, N)).astype(np.float32)
    y = (X[0] * X[1] + np.cos(X[2])).astype(np.float32)
    progs = _const_heavy_programs(rng, 600, d)
    refs = parity.references(progs, X, y)
    ds = beagle.Dataset(X, y)
    dp = beagle.DevicePrograms(progs)
    try:
        beagle.set_launch_config(keep_order=2)   # the packing kernel (it folds)
        folded = beagle.unpack_fitness(beagle.score_programs(dp, ds))
        fout, _ = beagle.eval_programs(dp, ds)
        fout = fout.cpu().numpy()
        beagle.set_launch_config(keep_order=1)   # each work item packs, unfolded
        plain = beagle.unpack_fitness(beagle.score_programs(dp, ds))
        pout, _ = beagle.eval_programs(dp, ds)
        pout = pout.cpu().numpy()
    finally:
        beagle.reset_launch_config()
    for a, b in zip(folded, plain):
        assert np.array_equal(a, b, equal_nan=True)
    assert np.array_equal(fout, pout, equal_nan=True)
    assert np.any(folded[2] & beagle.FLAG_INVALID) and not np.all(folded[2] & beagle.FLAG_INVALID)
    parity.check_fp32(folded, refs)
    ds.release()


@pytest.mark.parametrize("cases", [4, 8, 2])
def test_packing_kernel_same_bits_as_per_item_packing(cases):
    """Programs packed once per call by the packing kernel (length order, constant folding,
    the deep list filled by the packing kernel) give the bits of programs each work item packs
    itself: random programs of every operator, deep ones, register (COPY/PASTE) ones,
    constant-heavy ones, and malformed ones (flagged the same way)."""
    rng = np.random.default_rng(90 + cases)
    d, N = 3, 1500
    X = rng.uniform(-1.5, 1.5, (d, N)).astype(np.float32)
    y = (X[0] * X[1] - np.tanh(X[2])).astype(np.float32)
    parts = [S.gen_programs(rng, 300, 4, 90, d, unary=S.ALL_UNARY, binary=S.ALL_BINARY),
             _deep_population(rng, 200, d)[0], _const_heavy_programs(rng, 200, d),
             S.with_registers(S.gen_programs(rng, 200, 6, 60, d), 5, 0.5, 4)]
    C = S.CONST
    bad = S.from_token_lists([[(S.ADD, 0)], [(C, 1.0), (C, 2.0)], [(S.LOAD0 + 5, 0)],
                              [(C, 1.0)] * 33 + [(S.ADD, 0)] * 32,
                              [(C, 1.0), (C, 2.0), (S.ADD, 0), (S.ADD, 0)]])
    toks = [t for pr in parts + [bad] for t in (pr.program(p) for p in range(pr.P))]
    progs = S.from_token_lists([list(zip(o, c)) for o, c in toks])
    ds = beagle.Dataset(X, y)
    dp = beagle.DevicePrograms(progs)
    got = {}
    try:
        for mode in (1, 2):
            beagle.set_launch_config(cases_per_lane=cases, keep_order=mode)
            got[mode] = beagle.unpack_fitness(beagle.score_programs(dp, ds))
    finally:
        beagle.reset_launch_config()
    for a, b in zip(got[1], got[2]):
        assert np.array_equal(a, b, equal_nan=True)
    assert np.all(got[2][2][-5:] & beagle.FLAG_MALFORMED)
    ds.release()
