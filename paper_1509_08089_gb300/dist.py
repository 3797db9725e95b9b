"""Sharding a sample budget over ranks (one GPU per rank).

Samples are independent and keyed by their id, so a budget splits into
contiguous id ranges, each rank counts its range with its own graph replica,
and the only exchange is the sum of 2 x 22 integer counts -- exact for any
number of ranks.  Weak scaling: every rank draws ``budget`` samples, rank r
takes ids [r K_l, (r+1) K_l) of each sub-method l.
"""
from __future__ import annotations

from typing import Callable

import numpy as np

from . import (MOSS4, MOSS4MIN, NSLOTS, PATH5, T5, moss_finalize, moss_finalize_min, moss_sample_counts,
               result_dict)


def shard(total: int, rank: int, world: int) -> tuple[int, int]:
    """Contiguous split of [0, total) into world parts; the first
    total % world parts get one extra id.  Returns (first, count)."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank/world")
    base, extra = divmod(total, world)
    first = rank * base + min(rank, extra)
    return first, base + (1 if rank < extra else 0)


def sub_budgets(k: int, budget: int, mix: bool = False) -> list[tuple[int, int]]:
    """(method, samples) per sub-method for one estimate: K1 = K2 for k = 5
    (Sec. 5.1.5); with mix (k = 4), MOSS-4 and MOSS-4Min share the budget
    evenly (Sec. 4.2)."""
    if k == 4 and mix:
        return [(MOSS4, budget // 2), (MOSS4MIN, budget - budget // 2)]
    if k == 4:
        return [(MOSS4, budget)]
    return [(T5, budget // 2), (PATH5, budget - budget // 2)]


def weak_ranges(k: int, budget: int, rank: int, mix: bool = False) -> list[tuple[int, int, int]]:
    """(method, first, count) of rank ``rank`` when every rank draws ``budget``."""
    return [(m, rank * K, K) for m, K in sub_budgets(k, budget, mix)]


class DeviceShards:
    """The device side of :func:`estimate_weak`: this rank's counts in one
    device buffer (one row per sub-method), read back once."""

    def __init__(self, g, stream=None):
        import torch
        self.g, self.stream = g, stream
        self.stats = g.stats()
        self.buf = torch.zeros((2, NSLOTS), dtype=torch.int64, device=f"cuda:{g.device}")

    def has_weight(self, method: int) -> bool:
        return not (self.stats.gamma[method][0] == 0 and self.stats.gamma[method][1] == 0)

    def count(self, slot: int, method: int, first: int, count: int, seed: int):
        moss_sample_counts(self.g.handle, method, first, count, seed, self.buf[slot], self.stream)

    def counts(self) -> np.ndarray:
        return self.buf.cpu().numpy()

    def finalize(self, k: int, mix: bool, K: np.ndarray, hits: np.ndarray) -> dict:
        if mix:
            return result_dict(moss_finalize_min(self.g.handle, K, hits, self.stream))
        return result_dict(moss_finalize(self.g.handle, k, K, hits, self.stream))


def estimate_weak(g, k: int, budget: int, seed: int, rank: int, world: int,
                  allreduce: Callable[[np.ndarray], np.ndarray], stream=None, mix: bool = False,
                  shards=None) -> dict:
    """One weak-scaled estimate: this rank's counts, summed over ranks by
    ``allreduce`` (int64[2, 22] -> int64[2, 22]), then the finalize of the
    summed counts with K_l = per-rank count x world.  Methods whose total
    weight is zero draw nothing (as in the single call).  ``shards`` (default
    :class:`DeviceShards` of g) does the counting and the finalize; any
    object with the same four methods can stand in for it."""
    sh = shards if shards is not None else DeviceShards(g, stream)
    K = [0, 0]
    for slot, (m, first, count) in enumerate(weak_ranges(k, budget, rank, mix)):
        if not sh.has_weight(m):
            continue
        sh.count(slot, m, first, count, seed)
        K[slot] = count * world
    total = allreduce(sh.counts())
    return sh.finalize(k, mix, np.array(K, dtype=np.uint64), total.astype(np.uint64))
