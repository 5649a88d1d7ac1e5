"""Monte-Carlo ranking on the GPU (beagle_rank) against the oracle's, bit for bit: group and
child count of every individual, from MSE records (lower is better) and from the paper's
fitness records (higher is better, taxed by length), with invalid and timed-out individuals."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_2607_06731_gb300 import beagle, synth as S

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    yield


def _draws(rng, P):
    sample = rng.choice(P, 100, replace=False).astype(np.int64)
    u = rng.random(P).astype(np.float32)
    return sample, u


@pytest.mark.parametrize("P", [100, 1000, 1_000_003])
def test_rank_matches_the_oracle_on_records(P):
    rng = np.random.default_rng(P)
    rec = np.zeros((P, 3), np.float64)
    rec[:, 0] = np.round(rng.exponential(1.0, P), 2)              # mse, with ties
    rec[rng.random(P) < 0.03, 0] = np.inf                           # invalid programs
    rec[rng.random(P) < 0.01, 0] = np.nan                           # timed out
    sample, u = _draws(rng, P)
    dev = torch.from_numpy(rec).cuda()
    g, c = beagle.rank(dev, torch.from_numpy(sample).cuda(), torch.from_numpy(u).cuda(), "mse")
    torch.cuda.synchronize()
    og, oc = oracle.rank(-rec[:, 0], sample, u)
    assert np.array_equal(g.cpu().numpy(), og)
    assert np.array_equal(c.cpu().numpy(), oc)


def test_one_generation_score_then_rank():
    """A generation's device side: score (beagle_score, beagle_score_fit), then rank on the
    fitness records where they are; the oracle ranks the same keys."""
    pr = S.make_c1(P=4096)
    ds = beagle.Dataset(pr.X, pr.y)
    dp = beagle.DevicePrograms(pr.programs)
    rng = np.random.default_rng(9)
    sample, u = _draws(rng, dp.P)
    ts, tu = torch.from_numpy(sample).cuda(), torch.from_numpy(u).cuda()
    fit = beagle.score_programs(dp, ds)
    g, c = beagle.rank(fit, ts, tu, "mse")
    mse = beagle.unpack_fitness(fit)[0]
    og, oc = oracle.rank(-mse, sample, u)
    assert np.array_equal(g.cpu().numpy(), og) and np.array_equal(c.cpu().numpy(), oc)
    res = beagle.score_fit(dp, ds, beagle.FIT_STD, 10_000, -1.0)   # default length tax
    g, c = beagle.rank(res, ts, tu, "taxed_score")
    taxed = beagle.unpack_fit(res)["taxed_score"]
    og, oc = oracle.rank(taxed, sample, u)
    assert np.array_equal(g.cpu().numpy(), og) and np.array_equal(c.cpu().numpy(), oc)
    # the best group breeds most: about 4 children each
    assert c.cpu().numpy()[og == 9].mean() == pytest.approx(4.0)
    ds.release()
