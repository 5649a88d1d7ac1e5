"""Population sharding over several GPUs ("Hardware Optimized": a generation's work is spread
over every GPU of the machine). Each rank scores the contiguous range of programs that
beagle_shard_by_cost gives it -- nearly equal summed program lengths, every program running on
the same cases -- with its own copy of the dataset; the only exchange is gathering the fitness
records in order once every rank is done (one all-gather, torch.distributed)."""
from __future__ import annotations

import numpy as np

from . import beagle


def shard(progs, rank: int, world: int):
    """This rank's (start, stop) and program subset."""
    bounds = beagle.shard_by_cost(progs.lengths, world)
    a, b = int(bounds[rank]), int(bounds[rank + 1])
    return (a, b), progs.subset(np.arange(a, b))


def score_sharded(progs, score_fn, rank: int, world: int, dist=None):
    """Score a population split over `world` ranks: score_fn(subset) returns this rank's
    fitness records (a numpy array, one row per program); the records of every rank are
    gathered (dist.all_gather_object) and returned in program order on every rank."""
    (a, b), sub = shard(progs, rank, world)
    mine = np.asarray(score_fn(sub)) if b > a else None
    if dist is None or world == 1:
        return mine
    parts = [None] * world
    dist.all_gather_object(parts, (a, b, mine))
    parts.sort(key=lambda t: t[0])
    return np.concatenate([p[2] for p in parts if p[2] is not None])
