"""Parity of the MOSS-4Min path (Sec. 4.2, Algorithm 2) with the CPU oracle.

Bit-exact: the ordered lists, d_{v,u}, Gamma-check_v and its total, the
alias tables of sigma-check^(v) and pi-check, every per-sample tuple with its
class and c(s), every (class, c) count, for both probe strategies; the lists
cover the three sort tiers (at most 128 entries, at most 4096, longer -- the
hub graph's centre has 11,999 neighbours and needs two merge rounds).  FP64
estimates of the MOSS-4 + MOSS-4Min mix: relative 1e-9 (same arithmetic,
same order).
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import synth
import paper_1509_08089_gb300 as moss
from helpers import slot_twin

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

MASK = (1 << 4) | (1 << 5) | moss.TABLES_4MIN


def hub_graph():
    """Vertex 0 adjacent to all 11,999 others, plus 40,000 random edges."""
    rng = np.random.default_rng(4)
    n = 12_000
    a = rng.integers(1, n, size=40_000)
    b = rng.integers(1, n, size=40_000)
    return synth.from_edges(n, [(0, i) for i in range(1, n)] + list(zip(a.tolist(), b.tolist())))


def two_hubs():
    """Two adjacent hubs, each joined to the same 100,000 leaves, plus 50,000
    random leaf edges: the second hub's Gamma-check exceeds 2^32 and the hubs'
    degrees exceed 2^16, so the sampler takes its two-record path there."""
    rng = np.random.default_rng(8)
    leaves = 100_000
    edges = [(0, 1)] + [(h, i) for h in (0, 1) for i in range(2, leaves + 2)]
    edges += zip(rng.integers(2, leaves + 2, 50_000).tolist(), rng.integers(2, leaves + 2, 50_000).tolist())
    return synth.from_edges(leaves + 2, edges)


def decorated_diamond():
    return synth.from_edges(8, [(0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 4), (2, 5), (3, 6), (3, 7)])


GRAPHS = {
    "gnp12": lambda: synth.gnp(12, 0.45, 5),
    "diamond": decorated_diamond,
    "cl_n200": lambda: synth.chung_lu(200, 2.3, 6.0, 30.0, seed=7),
    "rgg2k": lambda: synth.rgg(2000, 12.0, seed=3),
    "cl_n2k": lambda: synth.workload("cl_n2k"),
    "hub12k": hub_graph,
    "twohub100k": two_hubs,
    "cl_n100k": lambda: synth.workload("cl_n100k"),
}

_cache = {}


def pair(name):
    if name not in _cache:
        rp, col = GRAPHS[name]()
        og = oracle.OracleGraph(rp, col)
        og.build_min()
        _cache[name] = (rp, col, og, moss.Graph(rp, col, device=0, k_mask=MASK))
    return _cache[name]


@pytest.fixture(scope="module", autouse=True)
def _cleanup():
    yield
    for rp, col, og, g in _cache.values():
        g.close()
    _cache.clear()


def gpu_records(g, first, count, seed):
    cls = torch.empty(count, dtype=torch.uint8, device="cuda")
    verts = torch.empty(count * 5, dtype=torch.int32, device="cuda")
    moss.moss_sample_records(g.handle, moss.MOSS4MIN, first, count, seed, cls, verts)
    torch.cuda.synchronize()
    return cls.cpu().numpy(), verts.cpu().numpy().view(np.uint32).reshape(count, 5)


def gpu_counts(g, first, count, seed, noalloc=False):
    c = torch.zeros(22, dtype=torch.int64, device="cuda")
    fn = moss.moss_sample_counts_noalloc if noalloc else moss.moss_sample_counts
    fn(g.handle, moss.MOSS4MIN, first, count, seed, c)
    torch.cuda.synchronize()
    return c.cpu().numpy().view(np.uint64)


def u64(lo, hi):
    return lo.astype(np.uint64) | (hi.astype(np.uint64) << np.uint64(32))


@pytest.mark.parametrize("name", list(GRAPHS))
def test_min_tables_bit_exact(name):
    rp, col, og, g = pair(name)
    n, nnz = og.n, og.nnz
    rl, rk, cthr, calias, gam = og.min_tables()
    vt = og.vertex_table(3)
    lst = moss.moss_table_export(g.handle, moss.TABLE_MIN_LIST, np.zeros((nnz, 2), dtype=np.uint32))
    assert np.array_equal(lst[:, 0], rl)
    deg = np.diff(rp.astype(np.int64))
    assert np.array_equal(lst[:, 1].astype(np.int64), deg[rl.astype(np.int64)])
    ms = moss.moss_table_export(g.handle, moss.TABLE_MIN_SLOT, np.zeros((nnz, 8), dtype=np.uint32))
    assert np.array_equal(u64(ms[:, 0], ms[:, 1]), cthr)
    assert np.array_equal(ms[:, 2], calias)
    assert np.array_equal(ms[:, 3], col)
    c64 = col.astype(np.int64)
    assert np.array_equal(ms[:, 4].astype(np.int64), rp.astype(np.int64)[c64])
    assert np.array_equal(ms[:, 5].astype(np.int64), deg[c64])
    assert np.array_equal(ms[:, 6].astype(np.uint64), rk)
    # d_{u,v}: the rank held by the twin slot (u -> v)
    slot = moss.moss_table_export(g.handle, moss.TABLE_SLOT, np.zeros((nnz, 8), dtype=np.uint32))
    twin_pos = rp.astype(np.int64)[c64] + slot_twin(slot)
    assert np.array_equal(ms[:, 7].astype(np.uint64), rk[twin_pos])
    mv = moss.moss_table_export(g.handle, moss.TABLE_MIN_VERT, np.zeros((n, 4), dtype=np.uint32))
    assert np.array_equal(mv[:, 0], rp[:-1].astype(np.uint32))
    assert np.array_equal(mv[:, 1].astype(np.int64), deg)
    gv = u64(mv[:, 2], mv[:, 3])
    assert [int(x) for x in gv] == gam
    gw = moss.moss_table_export(g.handle, moss.TABLE_MIN_GAMMA, np.zeros((n, 2), dtype=np.uint64))
    assert [int(a) | (int(b) << 64) for a, b in gw] == gam
    assert moss.moss_vertex_levels(g.handle, 3) == (vt["nh"], vt["TL"])
    seed = moss.moss_table_export(g.handle, moss.TABLE_MIN_SEED, np.zeros((n, 8), dtype=np.uint32))
    assert np.array_equal(u64(seed[:, 0], seed[:, 1]), vt["T"])
    assert np.array_equal(seed[:, 2], vt["alias"])
    assert np.array_equal(seed[:, 3], vt["self"])
    assert np.array_equal(seed[:, 4:8], mv[vt["alias"].astype(np.int64)])
    st = g.stats()
    assert (int(st.gamma[3][0]) | (int(st.gamma[3][1]) << 64)) == og.Gamma_min
    # pick records: the draw and both possible picks, from the oracle's tables
    pk = moss.moss_table_export(g.handle, moss.TABLE_MIN_PICK, np.zeros((nnz, 8), dtype=np.uint32))
    owner = np.repeat(np.arange(n, dtype=np.int64), deg)
    apos = rp.astype(np.int64)[owner] + calias.astype(np.int64)
    duv = rk[twin_pos].astype(np.int64)
    du = deg[c64]
    narrow = np.array([int(gam[v]) < (1 << 32) for v in range(n)], dtype=bool)[owner]
    small = (du < 0xFFFF) & (rk.astype(np.int64) < 0xFFFF) & (duv < 0xFFFF)
    fits = narrow & small & small[apos]
    expect = np.where(fits, du | (du[apos] << 16), 0xFFFFFFFF).astype(np.uint32)
    assert np.array_equal(pk[:, 7], expect)
    f = fits
    assert np.array_equal(pk[f, 0].astype(np.uint64), cthr[f])
    assert np.array_equal(pk[f, 1], col[f])
    assert np.array_equal(pk[f, 2].astype(np.int64), rp.astype(np.int64)[c64][f])
    dd = (rk.astype(np.int64) | (duv << 16)).astype(np.uint32)
    assert np.array_equal(pk[f, 3], dd[f])
    assert np.array_equal(pk[f, 4], col[apos][f])
    assert np.array_equal(pk[f, 5].astype(np.int64), rp.astype(np.int64)[c64][apos][f])
    assert np.array_equal(pk[f, 6], dd[apos][f])


RNGS = [("splitmix64", moss.RNG_SPLITMIX64, oracle.SPLITMIX64), ("philox4x32", moss.RNG_PHILOX4X32, oracle.PHILOX4X32)]


@pytest.mark.parametrize("rng", RNGS, ids=lambda r: r[0])
@pytest.mark.parametrize("name", list(GRAPHS))
def test_min_records_bit_exact(name, rng):
    _, lib_rng, orc_rng = rng
    rp, col, og, g = pair(name)
    if og.Gamma_min == 0:
        pytest.skip("no admissible tuple")
    first, count = (12_345, 100_003) if name != "cl_n100k" else (49_990_000, 20_011)
    seed = 0xBEEF
    ocnt, ocls, overts = og.run(oracle.MOSS4MIN, seed, count, first=first, record=True, rng=orc_rng)
    g.set_rng(lib_rng)
    try:
        for probe in (moss.PROBE_SEARCH, moss.PROBE_HASH, moss.PROBE_FILTER):
            g.set_probe(probe)
            cls, verts = gpu_records(g, first, count, seed)
            bad = np.nonzero(ocls != cls)[0]
            assert bad.size == 0, (probe, bad[:5], ocls[bad[:5]], cls[bad[:5]], overts[bad[:3]], verts[bad[:3]])
            assert np.array_equal(verts, overts), probe
            assert np.array_equal(gpu_counts(g, first, count, seed), ocnt), probe
    finally:
        g.set_rng(moss.RNG_SPLITMIX64)
        g.set_probe(moss.PROBE_AUTO)
    if name == "diamond":
        hit = [i for i in range(count) if set(overts[i, :4]) == {0, 1, 2, 3}]
        assert hit and all(overts[i, 4] == 3 for i in hit)


def test_min_shards_and_noalloc():
    rp, col, og, g = pair("cl_n2k")
    K, seed = 300_007, 5
    full = gpu_counts(g, 0, K, seed)
    a = 123_457
    assert np.array_equal(full, gpu_counts(g, 0, a, seed) + gpu_counts(g, a, K - a, seed))
    assert np.array_equal(full, gpu_counts(g, 0, K, seed, noalloc=True))
    assert np.array_equal(full, og.run(oracle.MOSS4MIN, seed, K))


def close(r, o, og):
    lam = float(og.Lambda3)
    for i in range(1, 7):
        tol_e = 1e-9 * (max(lam, 1.0) if i == 2 else max(abs(o["est"][i]), 1e-300))
        assert abs(r["est"][i] - o["est"][i]) <= tol_e, (i, r["est"][i], o["est"][i])
        tol_v = 1e-9 * max(abs(o["var"][i]), 1e-300) + (1e-9 * lam ** 2 / 1e6 if i == 2 else 0.0)
        assert abs(r["var"][i] - o["var"][i]) <= tol_v, (i, r["var"][i], o["var"][i])
        for l in range(2):
            assert abs(r["lam"][l][i] - o["lam"][l][i]) <= 1e-9, (i, l)
        assert abs(r["conc"][i] - o["conc"][i]) <= 1e-9 * max(abs(o["conc"][i]), 1e-300) + 1e-12
    assert abs(r["triangles"] - o["triangles"]) <= 1e-9 * max(abs(o["triangles"]), 1e-300)


@pytest.mark.parametrize("rng", RNGS, ids=lambda r: r[0])
@pytest.mark.parametrize("name", ["gnp12", "diamond", "cl_n200", "rgg2k", "cl_n2k", "hub12k"])
def test_estimate_min_matches_oracle(name, rng):
    _, lib_rng, orc_rng = rng
    rp, col, og, g = pair(name)
    K, Km, seed = 200_001, 150_003, 77
    g.set_rng(lib_rng)
    try:
        for probe in (moss.PROBE_SEARCH, moss.PROBE_HASH, moss.PROBE_FILTER):
            g.set_probe(probe)
            r = g.estimate_min(K, Km, seed)
            o = og.estimate_min(K, Km, seed, rng=orc_rng)
            assert tuple(r["K"]) == tuple(o["K"])
            ref4 = og.run(oracle.MOSS4, seed, K, rng=orc_rng) if og.Gamma[0] else np.zeros(22, np.uint64)
            refm = og.run(oracle.MOSS4MIN, seed, Km, rng=orc_rng) if og.Gamma_min else np.zeros(22, np.uint64)
            assert np.array_equal(r["hits"][0], ref4)
            assert np.array_equal(r["hits"][1], refm)
            close(r, o, og)
    finally:
        g.set_rng(moss.RNG_SPLITMIX64)
        g.set_probe(moss.PROBE_AUTO)


def test_finalize_min_and_covariance():
    rp, col, og, g = pair("cl_n2k")
    hits = np.zeros((2, 22), dtype=np.uint64)
    hits[0] = og.run(oracle.MOSS4, 3, 80_000)
    hits[1] = og.run(oracle.MOSS4MIN, 3, 60_000)
    o = oracle.finalize_moss4min(hits[0], hits[1], 80_000, 60_000, og.Gamma[0], og.Gamma_min, og.Lambda3)
    r = moss.result_dict(moss.moss_finalize_min(g.handle, [80_000, 60_000], hits))
    close(r, o, og)
    cov, r2 = moss.moss_finalize_min(g.handle, [80_000, 60_000], hits, covariance=True)
    close(moss.result_dict(r2), o, og)
    scale = np.abs(o["cov"]).max()
    assert np.allclose(cov, o["cov"], rtol=1e-9, atol=1e-9 * scale)
    # one sub-method only
    for K in ([80_000, 0], [0, 60_000]):
        o = oracle.finalize_moss4min(hits[0], hits[1], K[0], K[1], og.Gamma[0], og.Gamma_min, og.Lambda3)
        close(moss.result_dict(moss.moss_finalize_min(g.handle, K, hits)), o, og)


@pytest.mark.parametrize("family", ["c4", "complete", "star", "empty"])
def test_min_special_graphs(family):
    if family == "c4":
        rp, col = synth.cycle(4)
    elif family == "complete":
        rp, col = synth.complete(9)
    elif family == "star":
        rp, col = synth.star(7)
    else:
        rp, col = np.zeros(6, dtype=np.uint64), np.zeros(0, dtype=np.uint32)
    og = oracle.OracleGraph(rp, col)
    og.build_min()
    with moss.Graph(rp, col, k_mask=MASK) as g:
        r = g.estimate_min(10_001, 10_001, 11)
        o = og.estimate_min(10_001, 10_001, 11)
        assert tuple(r["K"]) == tuple(o["K"])
        close(r, o, og)
        if family == "c4":
            assert r["hits"][1][0] == 10_001 and r["est"][3] == pytest.approx(1.0)
        if family == "complete":
            assert int(r["hits"][1][oracle.min_slot(6, 3)]) == int(r["hits"][1].sum())
        if family in ("star", "empty"):
            assert r["K"][1] == 0
            with pytest.raises(moss.MossError):
                gpu_counts(g, 0, 10, 1)


def test_min_requires_its_tables():
    rp, col = synth.workload("cl_n2k")
    with moss.Graph(rp, col) as g:
        with pytest.raises(moss.MossError) as ei:
            gpu_counts(g, 0, 10, 1)
        assert ei.value.status == moss.MOSS_ESTATE
        with pytest.raises(moss.MossError) as ei:
            g.estimate_min(10, 10, 1)
        assert ei.value.status == moss.MOSS_ESTATE
        moss.moss_build_tables(g.handle, moss.TABLES_4MIN)
        with pytest.raises(moss.MossError):   # MOSS-4's tables went with the rebuild
            g.estimate_min(10, 10, 1)
        assert int(gpu_counts(g, 0, 1000, 1).sum()) <= 1000


def test_min_full_size():
    """MOSS-4Min at 5e7 samples on the 1M-edge graph: counts add up, the last
    samples match the oracle one by one, and an independent seed agrees with
    the mixed estimate within its variance."""
    rp, col, og, g = pair("cl_n100k")
    K = 50_000_000
    r = g.estimate_min(K, K, seed=42)
    assert tuple(r["K"]) == (K, K)
    assert int(r["hits"][0].sum()) == K
    assert int(r["hits"][1].sum()) <= K
    o = oracle.finalize_moss4min(r["hits"][0], r["hits"][1], K, K, og.Gamma[0], og.Gamma_min, og.Lambda3)
    close(r, o, og)
    cls, verts = gpu_records(g, K - 5000, 5000, 42)
    _, ocls, overts = og.run(oracle.MOSS4MIN, 42, 5000, first=K - 5000, record=True)
    assert np.array_equal(cls, ocls)
    assert np.array_equal(verts, overts)
    r2 = g.estimate_min(K, K, seed=43)
    for i in (1, 3, 4, 5, 6):
        sd = np.sqrt(r["var"][i] + r2["var"][i])
        assert abs(r["est"][i] - r2["est"][i]) <= 6 * sd + 1e-6 * abs(r["est"][i]), i
