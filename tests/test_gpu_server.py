"""The continuous-batching server: results are the same alone and in the mix.

Requests from several submitting threads (fixed budgets and target errors,
k = 4 and 5, several graphs) are served concurrently; each result must equal
moss_sample_estimate on the same graph with the request's final budget and
seed -- counts bit for bit, estimates exactly (same device finalize)."""
from __future__ import annotations

import threading

import numpy as np
import pytest

import oracle
import synth
import paper_1509_08089_gb300 as moss
from helpers import close_estimates

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pool_csrs():
    csrs = [synth.chung_lu(n, g, d, 60.0, seed=s)
            for n, g, d, s in ((800, 2.3, 6.0, 1), (3000, 2.6, 8.0, 2), (6000, 2.2, 10.0, 3))]
    csrs.append(synth.rgg(4000, 14.0, seed=4))
    graphs = [moss.Graph(rp, col) for rp, col in csrs]
    yield csrs, graphs
    for g in graphs:
        g.close()


@pytest.fixture(scope="module")
def pool(pool_csrs):
    return pool_csrs[1]


def submit_all(server, gids, plan, out, lock):
    for gi, k, budget, eps, seed in plan:
        rid = server.submit(gids[gi], k, budget=budget, target_rse=eps, seed=seed)
        with lock:
            out.append((rid, gi, k, seed))


@pytest.mark.parametrize("cfg", [dict(max_active=64, tick_samples=2_000_000, tile_samples=1024),
                                 dict(max_active=3, tick_samples=200_000, tile_samples=4096)])
def test_server_results_equal_solo_runs(pool, cfg):
    rng = np.random.default_rng(9)
    plans = []
    for t in range(4):
        plan = []
        for _ in range(10):
            gi = int(rng.integers(0, len(pool)))
            k = int(rng.choice([4, 5]))
            if rng.random() < 0.5:
                plan.append((gi, k, int(rng.integers(1_000, 500_000)), 0.0, int(rng.integers(1, 2**62))))
            else:
                plan.append((gi, k, 0, float(rng.uniform(0.02, 0.05)), int(rng.integers(1, 2**62))))
        plans.append(plan)
    subs, lock = [], threading.Lock()
    with moss.Server(min_budget=10_000, max_budget=2_000_000, pilot_samples=20_000, **cfg) as server:
        gids = [server.add_graph(g) for g in pool]
        threads = [threading.Thread(target=submit_all, args=(server, gids, p, subs, lock)) for p in plans]
        for th in threads:
            th.start()
        for th in threads:
            th.join()
        results = [(server.wait(rid, 300.0), gi, k, seed) for rid, gi, k, seed in subs]
        stats = server.stats()
    assert stats["completed"] == len(subs)
    for (r, st), gi, k, seed in results:
        solo = pool[gi].estimate(k, st["budget"], seed)
        assert tuple(r["K"]) == tuple(solo["K"])
        assert np.array_equal(r["hits"], solo["hits"])
        assert np.array_equal(r["est"], solo["est"])
        assert np.array_equal(r["var"], solo["var"])
        assert st["latency_s"] >= st["queue_s"] >= 0.0


def test_server_min_requests_equal_solo_runs():
    """MOSS-4 + MOSS-4Min requests served among plain ones equal
    moss_sample_estimate_min with the same budgets and seed."""
    mask = (1 << 4) | (1 << 5) | moss.TABLES_4MIN
    csrs = [synth.chung_lu(2500, 2.3, 8.0, 60.0, seed=7), synth.rgg(3000, 12.0, seed=8)]
    graphs = [moss.Graph(rp, col, k_mask=mask) for rp, col in csrs]
    try:
        with moss.Server(max_active=8, tick_samples=300_000, tile_samples=1024) as server:
            gids = [server.add_graph(g) for g in graphs]
            subs = []
            for j in range(6):
                gi = j % 2
                K, Km, seed = 40_000 + 9_000 * j, 30_000 + 7_000 * j, 100 + j
                subs.append(("min", gi, (K, Km, seed), server.submit_min(gids[gi], K, Km, seed=seed)))
                subs.append(("k5", gi, (K, seed), server.submit(gids[gi], 5, budget=K, seed=seed)))
            for kind, gi, args, rid in subs:
                r, st = server.wait(rid)
                solo = graphs[gi].estimate_min(*args) if kind == "min" else graphs[gi].estimate(5, *args)
                assert tuple(r["K"]) == tuple(solo["K"])
                assert np.array_equal(r["hits"], solo["hits"])
                assert np.array_equal(r["est"], solo["est"])
                assert np.array_equal(r["var"], solo["var"])
            with pytest.raises(moss.MossError):
                server.submit_min(gids[0], 0, 0)
    finally:
        for g in graphs:
            g.close()


def test_target_budget_meets_target(pool):
    """The budget is the rule applied to the pilot (the request's first
    50,000 ids), and every class with at least 10 pilot hits ends with a
    relative SE of at most eps sqrt((1/f - 1) / (1/f_pilot - 1)) -- eps itself
    when the final hit fraction f equals the pilot's (Theorem 3: the
    relative SE of a class is sqrt((1/f - 1) / K))."""
    eps, P = 0.02, 50_000
    with moss.Server(min_budget=1_000, max_budget=50_000_000, pilot_samples=P) as server:
        gid = server.add_graph(pool[2])
        rid = server.submit(gid, 4, target_rse=eps, seed=3)
        r, st = server.wait(rid)
    pilot = pool[2].estimate(4, P, 3)
    assert st["budget"] == moss.moss_budget_for_target(4, [P, 0], pilot["hits"], eps, 1_000, 50_000_000)
    K = r["K"][0]
    checked = 0
    for i in (1, 3, 4, 5, 6):
        mp = int(pilot["hits"][0][i])
        if mp < 10:
            continue
        fp, f = mp / P, int(r["hits"][0][i]) / K
        rse = np.sqrt(r["var"][i]) / r["est"][i]
        assert rse == pytest.approx(np.sqrt((1 / f - 1) / K), rel=1e-9), i
        assert rse <= eps * np.sqrt((1 / f - 1) / (1 / fp - 1)) * (1 + 1e-9), i
        checked += 1
    assert checked >= 3


def test_server_rejects_bad_requests(pool):
    with moss.Server() as server:
        gid = server.add_graph(pool[0])
        with pytest.raises(moss.MossError):
            server.submit(gid, 3, budget=100)
        with pytest.raises(moss.MossError):
            server.submit(gid + 5, 4, budget=100)
        with pytest.raises(moss.MossError):
            server.submit(gid, 4)          # neither budget nor target
        with pytest.raises(moss.MossError) as ei:
            server.submit_min(gid, 100, 100)   # MOSS-4Min tables not built
        assert ei.value.status == moss.MOSS_ESTATE
        rid = server.submit(gid, 4, budget=10_000, seed=1)
        server.wait(rid)
        with pytest.raises(moss.MossError):
            server.wait(rid)               # a request is waited for once


def test_served_results_match_oracle(pool_csrs):
    """Served results -- k = 4 and k = 5 with fixed budgets, k = 4 and k = 5
    with target errors (budget from the pilot), and a MOSS-4 + MOSS-4Min
    request on a graph drawing Philox words -- each against the oracle's
    whole path with the request's final budget and seed: counts bit for bit,
    estimates within 1e-9."""
    csrs, graphs = pool_csrs
    mask = (1 << 4) | (1 << 5) | moss.TABLES_4MIN
    rp_m, col_m = synth.chung_lu(2500, 2.3, 8.0, 60.0, seed=7)
    gmin = moss.Graph(rp_m, col_m, k_mask=mask, rng=moss.RNG_PHILOX4X32)    # served under Philox words
    try:
        with moss.Server(max_active=16, tick_samples=400_000, tile_samples=2048, min_budget=10_000,
                         max_budget=3_000_000, pilot_samples=20_000) as server:
            gids = [server.add_graph(g) for g in graphs]
            gid_m = server.add_graph(gmin)
            plan = [(2, 4, 700_001, 0.0, 11), (1, 5, 900_000, 0.0, 12), (0, 4, 0, 0.03, 13),
                    (3, 5, 0, 0.04, 14), (2, 5, 0, 0.05, 15)]
            subs = [(gi, k, seed, server.submit(gids[gi], k, budget=b, target_rse=eps, seed=seed))
                    for gi, k, b, eps, seed in plan]
            rid_m = server.submit_min(gid_m, 300_000, 200_000, seed=16)
            rid_t = server.submit_min(gid_m, target_rse=0.03, seed=18)     # budget from its pilot
            served = [(gi, k, seed, *server.wait(rid, 300.0)) for gi, k, seed, rid in subs]
            r_m, _ = server.wait(rid_m, 300.0)
            r_t, st_t = server.wait(rid_t, 300.0)
        assert sum(1 for _, _, _, _, st in served if st["budget"] not in (700_001, 900_000)) == 3
        for gi, k, seed, r, st in served:
            og = oracle.OracleGraph(*csrs[gi])
            o = og.estimate(k, st["budget"], seed)
            assert tuple(r["K"]) == tuple(o["K"])
            methods = (oracle.MOSS4,) if k == 4 else (oracle.T5, oracle.PATH5)
            for slot, method in enumerate(methods):
                K = o["K"][slot]
                ref = og.run(method, seed, K) if K else np.zeros(22, np.uint64)
                assert np.array_equal(r["hits"][slot], ref), (gi, k, slot)
            close_estimates(r, o, og, k)
        og = oracle.OracleGraph(rp_m, col_m)
        o = og.estimate_min(300_000, 200_000, 16, rng=oracle.PHILOX4X32)
        assert np.array_equal(r_m["hits"][0], og.run(oracle.MOSS4, 16, 300_000, rng=oracle.PHILOX4X32))
        assert np.array_equal(r_m["hits"][1], og.run(oracle.MOSS4MIN, 16, 200_000, rng=oracle.PHILOX4X32))
        for i in range(1, 7):
            tol = 1e-9 * (max(float(og.Lambda3), 1.0) if i == 2 else max(abs(o["est"][i]), 1e-300))
            assert abs(r_m["est"][i] - o["est"][i]) <= tol, i
        # the target-error MOSS-4 + MOSS-4Min request: K = floor(B/2), K-check = B - K
        K, Km = r_t["K"]
        assert K == st_t["budget"] // 2 and Km == st_t["budget"] - K and st_t["budget"] >= 20_000
        o = og.estimate_min(K, Km, 18, rng=oracle.PHILOX4X32)
        assert np.array_equal(r_t["hits"][0], og.run(oracle.MOSS4, 18, K, rng=oracle.PHILOX4X32))
        assert np.array_equal(r_t["hits"][1], og.run(oracle.MOSS4MIN, 18, Km, rng=oracle.PHILOX4X32))
        for i in range(1, 7):
            tol = 1e-9 * (max(float(og.Lambda3), 1.0) if i == 2 else max(abs(o["est"][i]), 1e-300))
            assert abs(r_t["est"][i] - o["est"][i]) <= tol, i
            if i != 2 and r_t["hits"][0][i] >= 200:       # well-sampled classes meet the target
                assert np.sqrt(r_t["var"][i]) / r_t["est"][i] <= 0.035, i
    finally:
        gmin.close()


def test_admission_waits_for_free_memory(pool):
    """With reserve_bytes above the device's free memory no request is
    admitted: it stays pending, and a short wait ends with MOSS_EBUSY."""
    free, _total = torch.cuda.mem_get_info()
    with moss.Server(reserve_bytes=free + (64 << 30)) as server:
        gid = server.add_graph(pool[0])
        rid = server.submit(gid, 4, budget=10_000, seed=1)
        with pytest.raises(moss.MossError) as ei:
            server.wait(rid, 0.3)
        assert ei.value.status == moss.MOSS_EBUSY
        st = server.stats()
        assert st["pending"] == 1 and st["active"] == 0 and st["completed"] == 0 and st["ticks"] == 0
