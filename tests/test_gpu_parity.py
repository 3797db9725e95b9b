"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Bit-exact: every table (vertex records, ACC, sigma alias tables, twins,
vertex alias tables, per-vertex weights, totals), every per-sample class and
vertex tuple, every count.  FP64 estimates: relative 1e-9 (the finalize is
the same arithmetic in the same order; eta_2 and n_2 are compared relative
to Lambda, since they are differences of large terms).
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import synth
import paper_1509_08089_gb300 as moss
from helpers import close_estimates, expected_slot_neighbour, oracle_counts, slot_twin

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

def hub_graph():
    """A star of 70,000 leaves, so one neighbour list holds 2^16 entries or
    more (slot records of that neighbour keep their twin in place of the list
    offset), with 60,000 random leaf-leaf edges and a second hub of 300."""
    rng = np.random.default_rng(11)
    leaves = 70_000
    edges = [(0, i) for i in range(1, leaves + 1)]
    edges += zip(rng.integers(1, leaves + 1, 60_000), rng.integers(1, leaves + 1, 60_000))
    edges += [(leaves + 1, int(x)) for x in rng.integers(1, leaves + 1, 300)]
    return synth.from_edges(leaves + 2, edges)


def circulant(n, offsets):
    """Vertex i adjacent to i +- o (mod n) for each offset o: a regular graph
    (degree 8 for (1, 2, 3, 4), 9 with n / 2 added) dense in triangles, so
    every class of both k and the collision paths occur often."""
    return synth.from_edges(n, [(i, (i + o) % n) for i in range(n) for o in offsets])


GRAPHS = {
    "gnp12": lambda: synth.gnp(12, 0.45, 5),
    "cl_n200": lambda: synth.chung_lu(200, 2.3, 6.0, 30.0, seed=7),
    "rgg2k": lambda: synth.rgg(2000, 12.0, seed=3),
    "cl_n2k": lambda: synth.workload("cl_n2k"),
    "cl_n100k": lambda: synth.workload("cl_n100k"),
    "hub70k": hub_graph,
    "circ8": lambda: circulant(300, (1, 2, 3, 4)),
    "circ9": lambda: circulant(300, (1, 2, 3, 4, 150)),
}

_cache = {}


def pair(name):
    if name not in _cache:
        rp, col = GRAPHS[name]()
        _cache[name] = (rp, col, oracle.OracleGraph(rp, col), moss.Graph(rp, col, device=0))
    return _cache[name]


@pytest.fixture(scope="module", autouse=True)
def _cleanup():
    yield
    for rp, col, og, g in _cache.values():
        g.close()
    _cache.clear()


def gpu_records(g, method, first, count, seed):
    cls = torch.empty(count, dtype=torch.uint8, device="cuda")
    verts = torch.empty(count * 5, dtype=torch.int32, device="cuda")
    moss.moss_sample_records(g.handle, method, first, count, seed, cls, verts)
    torch.cuda.synchronize()
    return cls.cpu().numpy(), verts.cpu().numpy().view(np.uint32).reshape(count, 5)


def gpu_counts(g, method, first, count, seed):
    c = torch.zeros(22, dtype=torch.int64, device="cuda")
    moss.moss_sample_counts(g.handle, method, first, count, seed, c)
    torch.cuda.synchronize()
    return c.cpu().numpy().view(np.uint64)


def u128(a):
    return [int(a[i, 0]) | (int(a[i, 1]) << 64) for i in range(a.shape[0])]


def check_vertex_table(g, og, l, vrec, table=None):
    """Two-level vertex table l against the oracle's, column by column:
    {T lo, T hi, alias, self} and the alias's vertex record; the level split."""
    n = og.n
    vt = og.vertex_table(l)
    assert moss.moss_vertex_levels(g.handle, l) == (vt["nh"], vt["TL"]), l
    seed = moss.moss_table_export(g.handle, table if table is not None else moss.TABLE_SEED0 + l,
                                  np.zeros((n, 8), dtype=np.uint32))
    Tg = seed[:, 0].astype(np.uint64) | (seed[:, 1].astype(np.uint64) << np.uint64(32))
    assert np.array_equal(Tg, vt["T"]), l
    assert np.array_equal(seed[:, 2], vt["alias"]), l
    assert np.array_equal(seed[:, 3], vt["self"]), l
    # the alias's vertex record rides in the second half of the column record
    assert np.array_equal(seed[:, 4:8], vrec[vt["alias"].astype(np.int64)]), l


@pytest.mark.parametrize("name", list(GRAPHS))
def test_tables_bit_exact(name):
    rp, col, og, g = pair(name)
    n, nnz = og.n, og.nnz
    deg, S, Q, gam = og.vertex()
    vert = moss.moss_table_export(g.handle, moss.TABLE_VERT, np.zeros((n, 4), dtype=np.uint32))
    assert np.array_equal(vert[:, 0], rp[:-1].astype(np.uint32))
    assert np.array_equal(vert[:, 1], deg.astype(np.uint32))
    assert np.array_equal(vert[:, 2], S.astype(np.uint32))
    thr, alias, acc = og.sigma_table()
    acc_g = moss.moss_table_export(g.handle, moss.TABLE_ACC, np.zeros(nnz, dtype=np.uint32))
    assert np.array_equal(acc_g, acc.astype(np.uint32))
    slot = moss.moss_table_export(g.handle, moss.TABLE_SLOT, np.zeros((nnz, 8), dtype=np.uint32))
    assert np.array_equal(slot[:, 0], col)
    assert np.array_equal(slot[:, 2], thr.astype(np.uint32))
    assert np.array_equal(slot[:, 3], alias)
    # twin: position of v in N_col
    owner = np.repeat(np.arange(n, dtype=np.int64), deg.astype(np.int64))
    c64 = col.astype(np.int64)
    pos = np.array([np.searchsorted(col[rp[x]:rp[x + 1]], v) for v, x in zip(owner, c64)], dtype=np.int64) \
        if nnz <= 200_000 else None
    twin = slot_twin(slot)
    if pos is not None:
        assert np.array_equal(twin, pos)
    else:  # large graph: check the defining property on all slots
        assert np.array_equal(col[rp.astype(np.int64)[c64] + twin].astype(np.int64), owner)
    # words 1 and 4: the neighbour's degree and list offset with the twin
    nb, off = expected_slot_neighbour(rp, col, twin)
    assert np.array_equal(slot[:, 1], nb)
    assert np.array_equal(slot[:, 4], off)
    # words 5..7 repeat the alias position's words 0, 1 and 4
    apos = rp.astype(np.int64)[owner] + slot[:, 3].astype(np.int64)
    assert np.array_equal(slot[:, 5], slot[apos, 0])
    assert np.array_equal(slot[:, 6], slot[apos, 1])
    assert np.array_equal(slot[:, 7], slot[apos, 4])
    for l in range(3):
        check_vertex_table(g, og, l, vert)
        gw = moss.moss_table_export(g.handle, moss.TABLE_GAMMA0 + l, np.zeros((n, 2), dtype=np.uint64))
        assert u128(gw) == gam[l]
    st = g.stats()
    for l in range(3):
        assert (int(st.gamma[l][0]) | (int(st.gamma[l][1]) << 64)) == og.Gamma[l]
    assert (int(st.lambda3[0]) | (int(st.lambda3[1]) << 64)) == og.Lambda3
    assert (int(st.lambda4[0]) | (int(st.lambda4[1]) << 64)) == og.Lambda4
    assert st.d_max == int(deg.max())


def filter_words(filter_hash, nnz):
    w = 1
    while w * 2 <= nnz // 8:
        w <<= 1
    return w


@pytest.mark.parametrize("name", ["gnp12", "rgg2k", "cl_n2k", "cl_n100k"])
def test_edge_filter_bits(name):
    """The filter holds exactly the bits of the edges (no false negatives) and
    rejects most non-edges."""
    from golden.sector_model import filter_hash, filter_mask
    rp, col, og, g = pair(name)
    g.set_probe(moss.PROBE_FILTER)
    nnz = len(col)
    W = filter_words(filter_hash, nnz)
    shift = np.uint64(64 - (W.bit_length() - 1))
    F = moss.moss_table_export(g.handle, moss.TABLE_FILTER, np.zeros(W, dtype=np.uint32))
    owner = np.repeat(np.arange(len(rp) - 1, dtype=np.uint64), np.diff(rp.astype(np.int64)))
    c64 = col.astype(np.uint64)
    keep = owner < c64
    h = filter_hash((owner[keep] << np.uint64(32)) | c64[keep])
    ref = np.zeros(W, dtype=np.uint32)
    np.bitwise_or.at(ref, (h >> shift).astype(np.int64), filter_mask(h))
    assert np.array_equal(F, ref)
    rng = np.random.default_rng(1)
    a = rng.integers(0, len(rp) - 1, 20000).astype(np.uint64)
    b = rng.integers(0, len(rp) - 1, 20000).astype(np.uint64)
    hh = filter_hash((np.minimum(a, b) << np.uint64(32)) | np.maximum(a, b))
    m = filter_mask(hh)
    passed = (F[(hh >> shift).astype(np.int64)] & m) == m
    if nnz >= 100_000:
        assert passed.mean() < 0.15
    g.set_probe(moss.PROBE_AUTO)


def hub_capacity(n):
    return min(8192, max(16, n // 16))


@pytest.mark.parametrize("name", ["gnp12", "cl_n200", "cl_n2k", "cl_n100k", "hub70k", "circ8"])
def test_hub_adjacency_bits(name):
    """The hubs are every vertex of degree >= D, D the smallest degree >= 1
    with at most H of them, listed in ascending id order, and their bitmap
    holds exactly their edges (hub i = the i-th hub)."""
    rp, col, og, g = pair(name)
    g.set_probe(moss.PROBE_FILTER)
    try:
        n = len(rp) - 1
        H = hub_capacity(n)
        deg = np.diff(rp.astype(np.int64))
        lst = moss.moss_table_export(g.handle, moss.TABLE_HUB_LIST, np.zeros(H, dtype=np.uint32))
        bits = moss.moss_table_export(g.handle, moss.TABLE_HUB_BITS, np.zeros((H * H + 31) // 32, dtype=np.uint32))
    finally:
        g.set_probe(moss.PROBE_AUTO)
    D = next(d for d in range(1, int(deg.max()) + 2) if (deg >= d).sum() <= H)
    hubs = lst[lst != 0xFFFFFFFF].astype(np.int64)
    assert np.array_equal(hubs, np.nonzero(deg >= D)[0])
    assert np.all(lst[len(hubs):] == 0xFFFFFFFF)
    assert (len(hubs) == 0) == (name == "circ8")     # a regular graph of more than H vertices has none
    index = np.full(n, -1, dtype=np.int64)
    index[hubs] = np.arange(len(hubs))
    want = np.zeros(H * H, dtype=bool)
    for i, v in enumerate(hubs):
        j = index[col[rp[v]:rp[v + 1]].astype(np.int64)]
        want[i * H + j[j >= 0]] = True
    got = np.unpackbits(bits.view(np.uint8), bitorder="little")[:H * H].astype(bool)
    assert np.array_equal(got, want)


RNGS = [("splitmix64", moss.RNG_SPLITMIX64, oracle.SPLITMIX64), ("philox4x32", moss.RNG_PHILOX4X32, oracle.PHILOX4X32)]


@pytest.mark.parametrize("rng", RNGS, ids=lambda r: r[0])
@pytest.mark.parametrize("name", ["gnp12", "cl_n200", "rgg2k", "cl_n2k", "cl_n100k", "hub70k", "circ8", "circ9"])
@pytest.mark.parametrize("method", [0, 1, 2])
def test_records_bit_exact(name, method, rng):
    _, lib_rng, orc_rng = rng
    rp, col, og, g = pair(name)
    if og.Gamma[method] == 0:
        pytest.skip("method has no sample on this graph")
    first, count = (12_345, 100_003) if name != "cl_n100k" else (49_990_000, 20_011)
    seed = 0xC0FFEE + method
    ocnt, ocls, overts = og.run(method, seed, count, first=first, record=True, rng=orc_rng)
    ncol = 4 if method == 0 else 5
    g.set_rng(lib_rng)
    try:
        for probe in (moss.PROBE_SEARCH, moss.PROBE_HASH, moss.PROBE_FILTER):
            g.set_probe(probe)
            cls, verts = gpu_records(g, method, first, count, seed)
            bad = np.nonzero(ocls != cls)[0]
            assert bad.size == 0, (probe, bad[:5], ocls[bad[:5]], cls[bad[:5]], overts[bad[:3]], verts[bad[:3]])
            assert np.array_equal(verts[:, :ncol], overts[:, :ncol])
            assert np.array_equal(gpu_counts(g, method, first, count, seed), ocnt), probe
    finally:
        g.set_rng(moss.RNG_SPLITMIX64)
        g.set_probe(moss.PROBE_AUTO)


@pytest.mark.parametrize("rng", RNGS, ids=lambda r: r[0])
@pytest.mark.parametrize("name", ["gnp12", "cl_n200", "rgg2k", "cl_n2k", "hub70k", "circ8"])
def test_counts_and_estimates(name, rng):
    _, lib_rng, orc_rng = rng
    rp, col, og, g = pair(name)
    budget, seed = 200_001, 99
    g.set_rng(lib_rng)
    try:
        for k, probe in ((4, moss.PROBE_SEARCH), (4, moss.PROBE_HASH), (4, moss.PROBE_FILTER),
                         (5, moss.PROBE_SEARCH), (5, moss.PROBE_HASH), (5, moss.PROBE_FILTER)):
            g.set_probe(probe)
            r = g.estimate(k, budget, seed)
            o = og.estimate(k, budget, seed, rng=orc_rng)
            if k == 4:
                ref = og.run(oracle.MOSS4, seed, budget, rng=orc_rng) if og.Gamma[0] else np.zeros(22, np.uint64)
                assert np.array_equal(r["hits"][0], ref)
            else:
                K1, K2 = budget // 2, budget - budget // 2
                ref1 = og.run(oracle.T5, seed, K1, rng=orc_rng) if og.Gamma[1] else np.zeros(22, np.uint64)
                ref2 = og.run(oracle.PATH5, seed, K2, rng=orc_rng) if og.Gamma[2] else np.zeros(22, np.uint64)
                assert np.array_equal(r["hits"][0], ref1)
                assert np.array_equal(r["hits"][1], ref2)
            assert tuple(r["K"]) == tuple(o["K"])
            close_estimates(r, o, og, k)
    finally:
        g.set_rng(moss.RNG_SPLITMIX64)
        g.set_probe(moss.PROBE_AUTO)


@pytest.mark.parametrize("name", ["cl_n200", "rgg2k", "cl_n2k", "hub70k"])
def test_small_split_draws_both_levels(name):
    """With a small split (the smallest from 3 up that leaves weight in both
    levels of a table) both levels of the vertex draws run: tables, records
    and counts against the oracle built with the same split."""
    rp, col = GRAPHS[name]()
    for split in range(3, 21):
        og = oracle.OracleGraph(rp, col, vsplit=split)
        if any(og.vertex_table(l)["nh"] > 0 and og.vertex_table(l)["TL"] > 0 for l in range(3)):
            break
    with moss.Graph(rp, col, vsplit=split) as g:
        vert = moss.moss_table_export(g.handle, moss.TABLE_VERT, np.zeros((og.n, 4), dtype=np.uint32))
        levels = []
        for l in range(3):
            check_vertex_table(g, og, l, vert)
            levels.append(og.vertex_table(l))
        assert any(v["nh"] > 0 and v["TL"] > 0 for v in levels)
        for method in (0, 1, 2):
            if og.Gamma[method] == 0:
                continue
            ocnt, ocls, overts = og.run(method, 77, 60_011, first=5, record=True)
            cls, verts = gpu_records(g, method, 5, 60_011, 77)
            assert np.array_equal(cls, ocls), method
            ncol = 4 if method == 0 else 5
            assert np.array_equal(verts[:, :ncol], overts[:, :ncol]), method
            assert np.array_equal(gpu_counts(g, method, 5, 60_011, 77), ocnt), method
        moss.moss_set_vertex_split(g.handle, split + 1)      # tables follow at the next build
        with pytest.raises(moss.MossError) as ei:
            g.estimate(4, 1000, 1)
        assert ei.value.status == moss.MOSS_ESTATE


def test_generator_setting():
    rp, col, og, g = pair("cl_n200")
    assert moss.moss_get_rng(g.handle) == moss.RNG_SPLITMIX64
    with pytest.raises(moss.MossError) as ei:
        moss.moss_set_rng(g.handle, 2)
    assert ei.value.status == moss.MOSS_EINVAL
    g.set_rng(moss.RNG_PHILOX4X32)
    assert moss.moss_get_rng(g.handle) == moss.RNG_PHILOX4X32
    a = g.estimate(5, 50_000, 3)
    g.set_rng(moss.RNG_SPLITMIX64)
    b = g.estimate(5, 50_000, 3)
    assert not np.array_equal(a["hits"], b["hits"])     # other words, other samples


@pytest.mark.parametrize("k", [4, 5])
def test_covariance_entry_matches_oracle(k):
    rp, col, og, g = pair("cl_n2k")
    hits = np.zeros((2, 22), dtype=np.uint64)
    if k == 4:
        hits[0] = og.run(oracle.MOSS4, 3, 80_000)
        K = [80_000, 0]
        o = oracle.finalize_moss4(hits[0], 80_000, og.Gamma[0], og.Lambda3)
    else:
        hits[0] = og.run(oracle.T5, 3, 50_000)
        hits[1] = og.run(oracle.PATH5, 3, 70_000)
        K = [50_000, 70_000]
        o = oracle.finalize_moss5(hits[0], hits[1], 50_000, 70_000, og.Gamma[1], og.Gamma[2], og.Lambda4)
    cov, r = moss.moss_covariance(g.handle, k, K, hits)
    close_estimates(r, o, og, k)
    scale = np.abs(o["cov"]).max()
    assert np.allclose(cov, o["cov"], rtol=1e-9, atol=1e-9 * scale)


def test_shards_add_up():
    rp, col, og, g = pair("cl_n2k")
    K, seed = 300_007, 5
    for method in (0, 1, 2):
        full = gpu_counts(g, method, 0, K, seed)
        a = 123_457
        parts = gpu_counts(g, method, 0, a, seed) + gpu_counts(g, method, a, K - a, seed)
        assert np.array_equal(full, parts)
        assert int(full.sum()) == K


def test_finalize_entry_matches_oracle():
    rp, col, og, g = pair("cl_n2k")
    hits = np.zeros((2, 22), dtype=np.uint64)
    hits[0] = og.run(oracle.T5, 3, 50_000)
    hits[1] = og.run(oracle.PATH5, 3, 70_000)
    r = moss.result_dict(moss.moss_finalize(g.handle, 5, [50_000, 70_000], hits))
    o = oracle.finalize_moss5(hits[0], hits[1], 50_000, 70_000, og.Gamma[1], og.Gamma[2], og.Lambda4)
    close_estimates(r, o, og, 5)


@pytest.mark.parametrize("family", ["cycle", "star", "complete", "empty", "isolated"])
def test_special_graphs(family):
    if family == "cycle":
        rp, col = synth.cycle(9)
    elif family == "star":
        rp, col = synth.star(7)
    elif family == "complete":
        rp, col = synth.complete(8)
    elif family == "empty":
        rp, col = np.zeros(6, dtype=np.uint64), np.zeros(0, dtype=np.uint32)
    else:  # a triangle plus isolated vertices
        rp, col = synth.from_edges(9, [(2, 5), (5, 7), (2, 7)])
    og = oracle.OracleGraph(rp, col)
    with moss.Graph(rp, col) as g:
        for k in (4, 5):
            r = g.estimate(k, 10_001, 11)
            o = og.estimate(k, 10_001, 11)
            assert tuple(r["K"]) == tuple(o["K"])
            methods = (0,) if k == 4 else (1, 2)
            for slot, method in enumerate(methods):
                K = r["K"][slot]
                ref = og.run(method, 11, K) if K else np.zeros(22, np.uint64)
                assert np.array_equal(r["hits"][slot], ref)
            close_estimates(r, o, og, k)
    if family == "cycle":
        assert r["est"][1] == pytest.approx(9.0, abs=1e-9)
    if family == "star":
        assert r["est"][2] == 35.0


def test_uint32_row_ptr_and_device_inputs():
    rp, col = synth.workload("cl_n2k")
    og = oracle.OracleGraph(rp, col)
    rp32 = torch.from_numpy(rp.astype(np.int32)).cuda()
    colt = torch.from_numpy(col.astype(np.int32)).cuda()
    with moss.Graph(rp32, colt) as g:
        r = g.estimate(4, 50_000, 1)
        assert np.array_equal(r["hits"][0], og.run(oracle.MOSS4, 1, 50_000))


def test_full_size_bench_config():
    """The benchmark's launch: k = 5, budget 1e8 on the 1M-edge graph."""
    rp, col, og, g = pair("cl_n100k")
    B = 100_000_000
    r = g.estimate(5, B, seed=42)
    K1, K2 = B // 2, B - B // 2
    assert tuple(r["K"]) == (K1, K2)
    assert int(r["hits"][0].sum()) == K1 and int(r["hits"][1].sum()) == K2
    from oracle.finalize import PHI5
    for i in range(1, 22):
        if PHI5[i - 1, 0] == 0:
            assert r["hits"][0][i] == 0
        if PHI5[i - 1, 1] == 0:
            assert r["hits"][1][i] == 0
    # all 2 x 22 counts of the full launch against the oracle's, run over the
    # same 1e8 sample ids on every host core
    om = [oracle_counts(og, method, 42, 0, K) for method, K in ((1, K1), (2, K2))]
    assert np.array_equal(r["hits"][0], om[0])
    assert np.array_equal(r["hits"][1], om[1])
    # so the device finalize of these counts is compared with the oracle's whole path
    o = oracle.finalize_moss5(om[0], om[1], K1, K2, og.Gamma[1], og.Gamma[2], og.Lambda4)
    close_estimates(r, o, og, 5)
    # the last samples of both sub-methods, one by one against the oracle
    for method, K in ((1, K1), (2, K2)):
        cls, verts = gpu_records(g, method, K - 5000, 5000, 42)
        _, ocls, overts = og.run(method, 42, 5000, first=K - 5000, record=True)
        assert np.array_equal(cls, ocls)
        assert np.array_equal(verts, overts)
    # under Philox words: the full launch's counts against the oracle's too
    g.set_rng(moss.RNG_PHILOX4X32)
    try:
        rp_ = g.estimate(5, B, seed=42)
    finally:
        g.set_rng(moss.RNG_SPLITMIX64)
    for slot, (method, K) in enumerate(((1, K1), (2, K2))):
        assert np.array_equal(rp_["hits"][slot], oracle_counts(og, method, 42, 0, K, rng=oracle.PHILOX4X32))
    # an independent seed agrees within the stated variances
    r2 = g.estimate(5, B, seed=43)
    for i in range(1, 22):
        sd = np.sqrt(r["var"][i] + r2["var"][i])
        assert abs(r["est"][i] - r2["est"][i]) <= 6 * sd + 1e-6 * abs(r["est"][i]), i
