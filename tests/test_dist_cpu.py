"""The N > 1 path on CPU: world_size-2 gloo ranks run
paper_1509_08089_gb300.dist.estimate_weak itself -- its id ranges, its
skipping of sub-methods with zero weight, its all-reduce of the counts and
its K per sub-method -- with the counting and the finalize done by the
oracle (no GPU here), and must reproduce the single-rank estimate of the
whole id range exactly."""
from __future__ import annotations

import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as tdist
import torch.multiprocessing as mp

from paper_1509_08089_gb300.dist import estimate_weak, shard, sub_budgets, weak_ranges


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


class OracleShards:
    """The counting and finalize of estimate_weak done by the oracle."""

    def __init__(self, og):
        self.og = og
        self.buf = np.zeros((2, 22), dtype=np.int64)
        self.calls = []

    def has_weight(self, method):
        return self.og.Gamma[method] > 0

    def count(self, slot, method, first, count, seed):
        self.calls.append((method, first, count))
        self.buf[slot] = self.og.run(method, seed, count, first=first).astype(np.int64)

    def counts(self):
        return self.buf

    def finalize(self, k, mix, K, hits):
        import oracle
        if k == 4:
            return {"K": tuple(int(x) for x in K), "hits": hits,
                    **oracle.finalize_moss4(hits[0], int(K[0]), self.og.Gamma[0], self.og.Lambda3)}
        return {"K": tuple(int(x) for x in K), "hits": hits,
                **oracle.finalize_moss5(hits[0], hits[1], int(K[0]), int(K[1]), self.og.Gamma[1], self.og.Gamma[2],
                                        self.og.Lambda4)}


GRAPH_CASES = {"cl300": lambda synth: synth.chung_lu(300, 2.3, 6.0, 40.0, seed=4),
               "cycle9": lambda synth: synth.cycle(9)}      # Gamma^(1) = 0: T-5 draws nothing


def _worker(rank, world, port, case, k, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    tdist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle
    import synth
    og = oracle.OracleGraph(*GRAPH_CASES[case](synth))
    sh = OracleShards(og)

    def allreduce(counts):
        t = torch.from_numpy(np.ascontiguousarray(counts))
        tdist.all_reduce(t)
        return t.numpy()

    r = estimate_weak(None, k, 20_001, 17, rank, world, allreduce, shards=sh)
    if rank == 0:
        out.put((r["K"], np.asarray(r["hits"]).copy(), np.asarray(r["est"]).copy(), sh.calls))
    tdist.barrier()
    tdist.destroy_process_group()


@pytest.mark.parametrize("case,k", [("cl300", 5), ("cl300", 4), ("cycle9", 5)])
def test_two_gloo_ranks_run_estimate_weak(case, k):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, case, k, q)) for r in range(2)]
    for p in procs:
        p.start()
    K, hits, est, calls = q.get(timeout=240)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    import oracle
    import synth
    og = oracle.OracleGraph(*GRAPH_CASES[case](synth))
    budget = 20_001
    # the single-rank run of both ranks' ids [0, 2 K_l) of every sub-method
    ref = og.estimate(k, 2 * budget, 17) if k == 4 else None
    subs = sub_budgets(k, budget)
    exp_K = tuple(2 * Kl if og.Gamma[m] > 0 else 0 for m, Kl in subs) + ((0,) if k == 4 else ())
    assert tuple(K) == exp_K
    for slot, (m, Kl) in enumerate(subs):
        want = og.run(m, 17, 2 * Kl).astype(np.uint64) if og.Gamma[m] > 0 else np.zeros(22, np.uint64)
        assert np.array_equal(hits[slot], want)
    # rank 0 counted ids [0, K_l) of each method with weight, nothing else
    assert calls == [(m, 0, Kl) for m, Kl in subs if og.Gamma[m] > 0]
    if k == 4:
        assert np.allclose(est, ref["est"], rtol=1e-12, atol=0)
    else:
        o = oracle.finalize_moss5(hits[0], hits[1], K[0], K[1], og.Gamma[1], og.Gamma[2], og.Lambda4)
        assert np.allclose(est, o["est"], rtol=1e-12, atol=0)
    if case == "cycle9":
        assert K[0] == 0 and est[1] == pytest.approx(9.0)    # eta_1 = 9 exactly from Path-5 alone
