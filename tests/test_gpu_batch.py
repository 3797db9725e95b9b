"""Batched persistent launch: many requests on many graphs in one kernel.

Each request must give exactly the counts and estimates of its solo
moss_sample_estimate (same sample ids, same finalize), whatever the tile size
and however often the captured launch is replayed; a few are also checked
against the oracle."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import synth
import paper_1509_08089_gb300 as moss

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def uneven_graphs(count: int, seed: int):
    """Half Chung-Lu (exponent 2.0-3.0), half 2-D RGG (mean degree 6-30),
    n from 500 to 5,000 -- a scaled-down version of the batched workload."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        n = int(rng.integers(500, 5000))
        if i % 2 == 0:
            gamma = float(rng.uniform(2.0, 3.0))
            dbar = float(rng.uniform(4.0, 12.0))
            out.append(synth.chung_lu(n, gamma, dbar, min(0.2 * n, 40 * dbar), seed=1000 + i))
        else:
            out.append(synth.rgg(n, float(rng.uniform(6.0, 30.0)), seed=2000 + i))
    return out


@pytest.fixture(scope="module")
def fleet():
    csrs = uneven_graphs(14, 3) + [synth.star(6), synth.cycle(9)]
    graphs = [moss.Graph(rp, col) for rp, col in csrs]
    yield csrs, graphs
    for g in graphs:
        g.close()


def requests(n_graphs: int, seed: int):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n_graphs):
        for _ in range(2):
            k = int(rng.choice([4, 5]))
            budget = int(rng.integers(10_000, 300_000))
            out.append((i, k, budget, int(rng.integers(1, 2**62))))
    return out


def same(a: dict, b: dict):
    assert tuple(a["K"]) == tuple(b["K"])
    assert np.array_equal(a["hits"], b["hits"])
    assert np.array_equal(a["est"], b["est"])
    assert np.array_equal(a["var"], b["var"])


def test_batch_equals_solo_runs(fleet):
    csrs, graphs = fleet
    reqs = requests(len(graphs), 11)
    with moss.Batch() as batch:
        for gi, k, budget, seed in reqs:
            batch.add(graphs[gi], k, budget, seed)
        assert len(batch) == len(reqs)
        res = batch.run()
        for (gi, k, budget, seed), r in zip(reqs, res):
            same(r, graphs[gi].estimate(k, budget, seed))
        # replay of the captured launch
        again = batch.run()
        for a, b in zip(res, again):
            same(a, b)
        # other tile sizes (ragged tiles everywhere) give the same results
        for tile in (32, 1000, 65536):
            batch.set_tile(tile)
            for a, b in zip(res, batch.run()):
                same(a, b)
        chosen = batch.tune()
        assert chosen in (1024, 4096, 16384, 65536)
        for a, b in zip(res, batch.run()):
            same(a, b)


def test_batch_against_oracle(fleet):
    csrs, graphs = fleet
    with moss.Batch() as batch:
        picks = [(0, 4, 40_001, 5), (1, 5, 30_003, 6), (14, 4, 1000, 7), (15, 5, 2000, 8)]
        for gi, k, budget, seed in picks:
            batch.add(graphs[gi], k, budget, seed)
        res = batch.run()
    for (gi, k, budget, seed), r in zip(picks, res):
        og = oracle.OracleGraph(*csrs[gi])
        if k == 4:
            ref = og.run(oracle.MOSS4, seed, budget) if og.Gamma[0] else np.zeros(22, np.uint64)
            assert np.array_equal(r["hits"][0], ref)
        else:
            K1, K2 = budget // 2, budget - budget // 2
            r1 = og.run(oracle.T5, seed, K1) if og.Gamma[1] else np.zeros(22, np.uint64)
            r2 = og.run(oracle.PATH5, seed, K2) if og.Gamma[2] else np.zeros(22, np.uint64)
            assert np.array_equal(r["hits"][0], r1)
            assert np.array_equal(r["hits"][1], r2)
    assert res[2]["est"][2] == 20.0          # star K_{1,6}: Gamma = 0, n_2 = C(6,3)
    assert res[3]["est"][1] == pytest.approx(9.0)   # cycle C_9: eta_1 = 9 exactly


def test_batch_mixes_generators():
    """Graphs drawing Philox words and graphs drawing SplitMix64 words in one
    launch: each request equals its solo run and the oracle's counts under
    its graph's generator."""
    csrs = uneven_graphs(4, 8)
    rngs = [moss.RNG_PHILOX4X32, moss.RNG_SPLITMIX64, moss.RNG_PHILOX4X32, moss.RNG_SPLITMIX64]
    graphs = [moss.Graph(rp, col, rng=r) for (rp, col), r in zip(csrs, rngs)]
    try:
        picks = [(i, k, 30_011 + 1000 * i, 70 + i) for i in range(4) for k in (4, 5)]
        with moss.Batch() as batch:
            for gi, k, budget, seed in picks:
                batch.add(graphs[gi], k, budget, seed)
            res = batch.run()
        for (gi, k, budget, seed), r in zip(picks, res):
            same(r, graphs[gi].estimate(k, budget, seed))
            og = oracle.OracleGraph(*csrs[gi])
            orng = oracle.PHILOX4X32 if rngs[gi] == moss.RNG_PHILOX4X32 else oracle.SPLITMIX64
            if k == 4:
                assert np.array_equal(r["hits"][0], og.run(oracle.MOSS4, seed, budget, rng=orng))
            else:
                K1, K2 = budget // 2, budget - budget // 2
                assert np.array_equal(r["hits"][0], og.run(oracle.T5, seed, K1, rng=orng))
                assert np.array_equal(r["hits"][1], og.run(oracle.PATH5, seed, K2, rng=orng))
    finally:
        for g in graphs:
            g.close()


def test_batch_min_requests_equal_solo_runs():
    """MOSS-4 + MOSS-4Min requests, mixed with plain k = 4 and 5 requests in
    one batch, equal moss_sample_estimate_min (and the oracle's counts)."""
    mask = (1 << 4) | (1 << 5) | moss.TABLES_4MIN
    csrs = uneven_graphs(6, 5) + [synth.complete(7)]
    graphs = [moss.Graph(rp, col, k_mask=mask) for rp, col in csrs]
    try:
        picks = [(i, 20_000 + 1_000 * i, 15_000 + 700 * i, 31 + i) for i in range(len(graphs))]
        with moss.Batch() as batch:
            for gi, K, Km, seed in picks:
                batch.add_min(graphs[gi], K, Km, seed)
                batch.add(graphs[gi], 5, K, seed)
            res = batch.run()
            for tile in (100, 4096):
                batch.set_tile(tile)
                for a, b in zip(res, batch.run()):
                    same(a, b)
        for j, (gi, K, Km, seed) in enumerate(picks):
            r = res[2 * j]
            same(r, graphs[gi].estimate_min(K, Km, seed))
            assert np.array_equal(r["lam"], graphs[gi].estimate_min(K, Km, seed)["lam"])
            same(res[2 * j + 1], graphs[gi].estimate(5, K, seed))
        og = oracle.OracleGraph(*csrs[0])
        og.build_min()
        gi, K, Km, seed = picks[0]
        assert np.array_equal(res[0]["hits"][1], og.run(oracle.MOSS4MIN, seed, Km))
    finally:
        for g in graphs:
            g.close()


def test_batch_rejects_unbuilt_graph_and_handles_empty():
    rp, col = synth.cycle(10)
    with moss.Graph(rp, col, k_mask=1 << 4) as g, moss.Batch() as batch:
        assert batch.run() == []
        with pytest.raises(moss.MossError) as ei:
            batch.add(g, 5, 100, 1)
        assert ei.value.status == moss.MOSS_ESTATE
        with pytest.raises(moss.MossError) as ei:
            batch.add_min(g, 100, 100, 1)
        assert ei.value.status == moss.MOSS_ESTATE
        batch.add(g, 4, 100, 1)
        assert batch.run()[0]["est"][1] == pytest.approx(10.0)


def test_every_tuner_setting_leaves_results_unchanged(fleet):
    """Each launch setting the autotuner chooses among -- threads per block,
    resident blocks per SM, each graph's probe strategy -- and the tuned
    choice itself give every request exactly its solo result."""
    csrs, graphs = fleet
    filt = [moss.Graph(rp, col, probe=moss.PROBE_FILTER) for rp, col in csrs[:4]]     # all three strategies
    srch = [moss.Graph(rp, col, probe=moss.PROBE_SEARCH) for rp, col in csrs[4:6]]    # list search only
    pool = graphs + filt + srch
    try:
        reqs = requests(len(pool), 17)
        solo = [pool[gi].estimate(k, budget, seed) for gi, k, budget, seed in reqs]
        with moss.Batch() as batch:
            for gi, k, budget, seed in reqs:
                batch.add(pool[gi], k, budget, seed)
            batch.set_tile(2048)
            for threads in (128, 256, 512):
                for per_sm in (1, 0):
                    batch.set_launch(threads, per_sm)
                    for a, b in zip(solo, batch.run()):
                        same(b, a)
            batch.set_launch(256, 0)
            for strategy in (moss.PROBE_SEARCH, moss.PROBE_HASH, moss.PROBE_FILTER):
                for g in pool:
                    try:
                        batch.set_probe(g, strategy)
                    except moss.MossError as e:       # the graph lacks that strategy's tables
                        assert e.status == moss.MOSS_ESTATE
                        assert strategy != moss.PROBE_SEARCH
                for a, b in zip(solo, batch.run()):
                    same(b, a)
            with pytest.raises(moss.MossError) as ei:
                batch.set_probe(srch[0], moss.PROBE_HASH)
            assert ei.value.status == moss.MOSS_ESTATE
            with pytest.raises(moss.MossError):
                batch.set_launch(100, 0)
            for g in pool:
                batch.set_probe(g, moss.PROBE_AUTO)
            chosen = batch.tune()
            t = batch.tuning()
            assert t["tuned"] == 1 and t["tile_samples"] == chosen
            assert t["threads_per_block"] in (128, 256, 512) and t["blocks_per_sm"] >= 1
            assert t["graphs"] == len(pool)
            # every graph that drew samples got a strategy it has tables for
            assert len(pool) - 1 <= t["graphs_search"] + t["graphs_hash"] + t["graphs_filter"] <= len(pool)
            assert t["graphs_filter"] <= len(filt) and t["graphs_search"] >= len(srch)
            for a, b in zip(solo, batch.run()):
                same(b, a)
    finally:
        for g in filt + srch:
            g.close()


def test_batch_on_two_level_graphs():
    """A graph of 2^14 vertices or more has two-level vertex tables by
    default; its solo launches run the L1-streaming sampler instances and the
    batch kernel the plain ones.  Both must give the oracle's counts."""
    csrs = [synth.chung_lu(20_000, 2.2, 10.0, 800.0, seed=77), synth.chung_lu(1_500, 2.5, 6.0, 120.0, seed=78)]
    graphs = [moss.Graph(rp, col) for rp, col in csrs]
    try:
        assert moss.moss_vertex_levels(graphs[0].handle, 1)[0] > 0
        picks = [(0, 5, 60_001, 91), (0, 4, 40_003, 92), (1, 5, 20_001, 93)]
        with moss.Batch() as batch:
            for gi, k, budget, seed in picks:
                batch.add(graphs[gi], k, budget, seed)
            res = batch.run()
        for (gi, k, budget, seed), r in zip(picks, res):
            same(r, graphs[gi].estimate(k, budget, seed))
            og = oracle.OracleGraph(*csrs[gi])
            if k == 4:
                assert np.array_equal(r["hits"][0], og.run(oracle.MOSS4, seed, budget))
            else:
                K1, K2 = budget // 2, budget - budget // 2
                assert np.array_equal(r["hits"][0], og.run(oracle.T5, seed, K1))
                assert np.array_equal(r["hits"][1], og.run(oracle.PATH5, seed, K2))
    finally:
        for g in graphs:
            g.close()
