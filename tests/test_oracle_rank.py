"""Pins of the oracle's Monte-Carlo ranking (oracle_rank): the overview's "Monte-Carlo Ranking"
and Table 2, against a hand-worked population, Table 2's expected children and a numpy
restatement (sort, searchsorted)."""
from __future__ import annotations

import numpy as np

import oracle


def test_hand_worked_groups():
    """Keys 0..199, the even ones sampled: thresholds 20, 40, ..., 180, so key p sits in
    group min(9, p // 20)."""
    key = np.arange(200, dtype=np.float64)
    sample = np.arange(0, 200, 2)
    g, c = oracle.rank(key, sample, np.full(200, 0.5, np.float32))
    assert np.array_equal(g, np.minimum(9, np.arange(200) // 20))
    # u = 0.5: floor(E) + (0.5 < frac(E))
    want = {0: 0, 1: 0, 2: 0, 3: 0, 4: 0, 5: 0, 6: 1, 7: 1, 8: 2, 9: 4}
    assert np.array_equal(c, [want[int(x)] for x in g])
    g0, c0 = oracle.rank(key, sample, np.zeros(200, np.float32))    # u = 0: every fraction wins
    want0 = {0: 1, 1: 1, 2: 1, 3: 1, 4: 1, 5: 1, 6: 1, 7: 2, 8: 3, 9: 4}
    assert np.array_equal(c0, [want0[int(x)] for x in g0])


def test_expected_children_follow_table_2():
    rng = np.random.default_rng(1)
    P = 400_000
    key = rng.standard_normal(P)
    sample = rng.choice(P, 100, replace=False)
    g, c = oracle.rank(key, sample, rng.random(P).astype(np.float32))
    for k, e in enumerate(oracle.TABLE2_CHILDREN):
        sel = g == k
        if sel.sum() < 2000:
            continue
        sd = np.sqrt(e * (1 - e % 1) if e % 1 else 0.0) / np.sqrt(sel.sum()) + 1e-12
        assert abs(c[sel].mean() - e) <= 5 * max(sd, np.sqrt(0.25 / sel.sum())), (k, c[sel].mean(), e)


def test_matches_a_numpy_restatement_with_ties_and_nan():
    rng = np.random.default_rng(2)
    P = 50_000
    key = np.round(rng.standard_normal(P), 1)          # many ties
    key[rng.random(P) < 0.05] = np.nan                 # timed-out or invalid individuals
    key[rng.random(P) < 0.05] = -np.inf
    u = rng.random(P).astype(np.float32)
    for trial in range(5):
        sample = rng.choice(P, 100, replace=False)
        g, c = oracle.rank(key, sample, u)
        s = key[sample]
        s = np.concatenate([s[np.isnan(s)], np.sort(s[~np.isnan(s)])])   # NaN first
        thr = s[10:100:10]
        ref = np.zeros(P, np.int64)
        for t in thr:
            if not np.isnan(t):
                with np.errstate(invalid="ignore"):
                    ref += (key >= t) & ~np.isnan(key)
        assert np.array_equal(g, ref)
        e = np.array(oracle.TABLE2_CHILDREN)[ref]
        assert np.array_equal(c, np.floor(e).astype(np.int64) +
                              (u.astype(np.float64) < e - np.floor(e)))
