"""The N > 1 path on CPU: world_size-2 gloo ranks shard sample ids with
paper_1509_08089_gb300.dist, count their shards (with the oracle: no GPU
here), all-reduce the counts, and must reproduce the single-rank counts of the
whole id range exactly."""
from __future__ import annotations

import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as tdist
import torch.multiprocessing as mp

from paper_1509_08089_gb300.dist import shard, sub_budgets, weak_ranges


def test_shard_partitions_exactly():
    for total in (0, 1, 7, 100, 1001):
        for world in (1, 2, 3, 8):
            parts = [shard(total, r, world) for r in range(world)]
            assert parts[0][0] == 0
            for (f0, c0), (f1, _c1) in zip(parts, parts[1:]):
                assert f0 + c0 == f1
            assert sum(c for _, c in parts) == total
            assert max(c for _, c in parts) - min(c for _, c in parts) <= 1


def test_weak_ranges_are_disjoint():
    seen = set()
    for r in range(4):
        for m, first, count in weak_ranges(5, 1001, r):
            for s in (first, first + count - 1):
                assert (m, s) not in seen
                seen.add((m, s))
    assert sub_budgets(5, 1001) == [(1, 500), (2, 501)]


def _free_port() -> int:
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    tdist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle
    import synth
    rp, col = synth.chung_lu(300, 2.3, 6.0, 40.0, seed=4)
    og = oracle.OracleGraph(rp, col)
    budget = 20_001
    counts = np.zeros((2, 22), dtype=np.int64)
    for slot, (m, first, count) in enumerate(weak_ranges(5, budget, rank)):
        counts[slot] = og.run(m, 17, count, first=first).astype(np.int64)
    t = torch.from_numpy(counts)
    tdist.all_reduce(t)
    if rank == 0:
        out.put(t.numpy().copy())
    tdist.barrier()
    tdist.destroy_process_group()


def test_two_gloo_ranks_sum_to_single_rank():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = q.get(timeout=240)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    import oracle
    import synth
    rp, col = synth.chung_lu(300, 2.3, 6.0, 40.0, seed=4)
    og = oracle.OracleGraph(rp, col)
    budget = 20_001
    ref = np.zeros((2, 22), dtype=np.int64)
    for slot, (m, K) in enumerate(sub_budgets(5, budget)):
        ref[slot] = og.run(m, 17, 2 * K).astype(np.int64)   # ids [0, 2K) = both ranks
    assert np.array_equal(got, ref)
