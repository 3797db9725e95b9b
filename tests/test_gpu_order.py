"""Degree-ordered loads (MOSS_ORDER_DEGREE) through the C ABI.

The renumbering is integer work and is compared bit for bit with its numpy
statement (helpers.degree_order): the id map, the renumbered row offsets and
lists.  The samplers then run on a graph the oracle also gets, renumbered by
that numpy statement: tables, per-sample classes, counts and estimates are
the oracle's on the renumbered CSR, and records come back in input ids
(the oracle's vertices mapped through the id map).  Invalid inputs are
rejected as an input-order load rejects them."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import synth
import paper_1509_08089_gb300 as moss
from helpers import close_estimates, degree_order, oracle_counts

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

MASK = (1 << 4) | (1 << 5) | moss.TABLES_4MIN


def hub_graph():
    """A star of 70,000 leaves with 60,000 random leaf-leaf edges and a second
    hub of 300: one list far longer than a warp's round, many lists of 1-3."""
    rng = np.random.default_rng(11)
    leaves = 70_000
    edges = [(0, i) for i in range(1, leaves + 1)]
    edges += zip(rng.integers(1, leaves + 1, 60_000), rng.integers(1, leaves + 1, 60_000))
    edges += [(leaves + 1, int(x)) for x in rng.integers(1, leaves + 1, 300)]
    return synth.from_edges(leaves + 2, edges)


GRAPHS = {
    "gnp12": lambda: synth.gnp(12, 0.45, 5),
    "cl_n200": lambda: synth.chung_lu(200, 2.3, 6.0, 30.0, seed=7),
    "rgg2k": lambda: synth.rgg(2000, 12.0, seed=3),
    "cl_n2k": lambda: synth.workload("cl_n2k"),
    "cl_n100k": lambda: synth.workload("cl_n100k"),   # 13 chunks of 8,192 vertices, the last ragged
    "hub70k": hub_graph,
    "isolated": lambda: synth.from_edges(37, [(2, 5), (5, 7), (2, 7), (30, 36), (7, 30)]),
}

_cache = {}


def quad(name):
    if name not in _cache:
        rp, col = GRAPHS[name]()
        order, nrp, ncol = degree_order(rp, col)
        og = oracle.OracleGraph(nrp, ncol)
        og.build_min()
        g = moss.Graph(rp, col, k_mask=MASK, order=moss.ORDER_DEGREE)
        _cache[name] = (rp, col, order, nrp, ncol, og, g)
    return _cache[name]


@pytest.fixture(scope="module", autouse=True)
def _cleanup():
    yield
    for v in _cache.values():
        v[-1].close()
    _cache.clear()


def records(g, method, first, count, seed):
    cls = torch.empty(count, dtype=torch.uint8, device="cuda")
    verts = torch.empty(count * 5, dtype=torch.int32, device="cuda")
    moss.moss_sample_records(g.handle, method, first, count, seed, cls, verts)
    torch.cuda.synchronize()
    return cls.cpu().numpy(), verts.cpu().numpy().view(np.uint32).reshape(count, 5)


def counts(g, method, first, count, seed):
    c = torch.zeros(22, dtype=torch.int64, device="cuda")
    moss.moss_sample_counts(g.handle, method, first, count, seed, c)
    torch.cuda.synchronize()
    return c.cpu().numpy().view(np.uint64)


@pytest.mark.parametrize("name", list(GRAPHS))
def test_renumbering_bit_exact(name):
    rp, col, order, nrp, ncol, og, g = quad(name)
    n, nnz = len(rp) - 1, len(col)
    got = moss.moss_table_export(g.handle, moss.TABLE_ORDER, np.zeros(n, dtype=np.uint32))
    assert np.array_equal(got, order)
    vert = moss.moss_table_export(g.handle, moss.TABLE_VERT, np.zeros((n, 4), dtype=np.uint32))
    assert np.array_equal(vert[:, 0], nrp[:-1].astype(np.uint32))
    assert np.array_equal(vert[:, 1], np.diff(nrp).astype(np.uint32))
    deg, S, Q, gam = og.vertex()
    assert np.array_equal(vert[:, 2], S.astype(np.uint32))
    slot = moss.moss_table_export(g.handle, moss.TABLE_SLOT, np.zeros((nnz, 8), dtype=np.uint32))
    assert np.array_equal(slot[:, 0], ncol)
    thr, alias, acc = og.sigma_table()
    assert np.array_equal(slot[:, 2], thr.astype(np.uint32))
    assert np.array_equal(slot[:, 3], alias)
    st = g.stats()
    for l in range(3):
        assert (int(st.gamma[l][0]) | (int(st.gamma[l][1]) << 64)) == og.Gamma[l]
    # the totals are those of the input graph too (relabelling invariance)
    base = oracle.OracleGraph(rp, col)
    assert base.Gamma == og.Gamma and base.Lambda3 == og.Lambda3 and base.Lambda4 == og.Lambda4


@pytest.mark.parametrize("name", list(GRAPHS))
@pytest.mark.parametrize("method", [0, 1, 2, 3])
def test_records_in_input_ids(name, method):
    rp, col, order, nrp, ncol, og, g = quad(name)
    if (og.Gamma_min if method == 3 else og.Gamma[method]) == 0:
        pytest.skip("method has no sample on this graph")
    first, count = (12_345, 50_003) if name != "cl_n100k" else (49_990_000, 20_011)
    seed = 0xD00D + method
    ocnt, ocls, overts = og.run(method, seed, count, first=first, record=True)
    words = 5 if method in (1, 2) else 4
    for probe in (moss.PROBE_SEARCH, moss.PROBE_HASH, moss.PROBE_FILTER):
        g.set_probe(probe)
        try:
            cls, verts = records(g, method, first, count, seed)
            bad = np.nonzero(ocls != cls)[0]
            assert bad.size == 0, (probe, bad[:5])
            assert np.array_equal(verts[:, :words], order[overts[:, :words].astype(np.int64)]), probe
            if method == 3:   # c(s) is not a vertex
                assert np.array_equal(verts[:, 4], overts[:, 4]), probe
            assert np.array_equal(counts(g, method, first, count, seed), ocnt), probe
        finally:
            g.set_probe(moss.PROBE_AUTO)


@pytest.mark.parametrize("name", ["gnp12", "cl_n200", "rgg2k", "cl_n2k", "hub70k", "isolated"])
def test_estimates_match_oracle(name):
    rp, col, order, nrp, ncol, og, g = quad(name)
    budget, seed = 200_001, 99
    for k in (4, 5):
        r = g.estimate(k, budget, seed)
        o = og.estimate(k, budget, seed)
        assert tuple(r["K"]) == tuple(o["K"])
        methods = (0,) if k == 4 else (1, 2)
        for s, method in enumerate(methods):
            K = r["K"][s]
            ref = og.run(method, seed, K) if K else np.zeros(22, np.uint64)
            assert np.array_equal(r["hits"][s], ref)
        close_estimates(r, o, og, k)


def test_input_order_map_is_identity():
    rp, col = synth.workload("cl_n2k")
    with moss.Graph(rp, col) as g:
        got = moss.moss_table_export(g.handle, moss.TABLE_ORDER, np.zeros(len(rp) - 1, dtype=np.uint32))
        assert np.array_equal(got, np.arange(len(rp) - 1, dtype=np.uint32))


def test_device_inputs_and_uint32_row_ptr():
    """Lists read in place from device memory, 32-bit row offsets."""
    rp, col = synth.workload("cl_n2k")
    order, nrp, ncol = degree_order(rp, col)
    rp32 = torch.from_numpy(rp.astype(np.int32)).cuda()
    colt = torch.from_numpy(col.astype(np.int32)).cuda()
    og = oracle.OracleGraph(nrp, ncol)
    with moss.Graph(rp32, colt, order=moss.ORDER_DEGREE) as g:
        got = moss.moss_table_export(g.handle, moss.TABLE_ORDER, np.zeros(len(rp) - 1, dtype=np.uint32))
        assert np.array_equal(got, order)
        r = g.estimate(4, 50_000, 1)
        assert np.array_equal(r["hits"][0], og.run(oracle.MOSS4, 1, 50_000))


def _csr(lists):
    rp = np.zeros(len(lists) + 1, dtype=np.uint64)
    for i, l in enumerate(lists):
        rp[i + 1] = rp[i] + len(l)
    return rp, np.array([x for l in lists for x in l], dtype=np.uint32)


@pytest.mark.parametrize("lists,word", [
    ([[1], [], [0]], "reverse"),
    ([[2, 1], [0], [0]], "increasing"),
    ([[0, 1], [0, 1]], "self loop"),
    ([[1, 1], [0, 0]], "increasing"),
    ([[5], [0]], "n"),
    ([list(range(2, 42)) + [1]] + [[0]] * 41, "increasing"),   # a long list out of order
    ([list(range(1, 40)) + [77, 78]] + [[0]] * 39, "n"),       # a long list with ids >= n
])
def test_invalid_csr_rejected(lists, word):
    rp, col = _csr(lists)
    with pytest.raises(moss.MossError) as ei:
        moss.moss_graph_load_csr(rp, col, order=moss.ORDER_DEGREE)
    assert ei.value.status == moss.MOSS_EGRAPH
    assert word in str(ei.value)


def test_bad_row_ptr_rejected():
    rp = np.array([0, 3, 2, 4], dtype=np.uint64)
    col = np.array([1, 2, 0, 0], dtype=np.uint32)
    with pytest.raises(moss.MossError) as ei:
        moss.moss_graph_load_csr(rp, col, order=moss.ORDER_DEGREE)
    assert ei.value.status == moss.MOSS_EGRAPH and "row_ptr" in str(ei.value)
    with pytest.raises(moss.MossError) as ei:
        moss.moss_graph_load_csr(rp, col, order=7)
    assert ei.value.status == moss.MOSS_EINVAL


# ------------------------------------------------------------ full size ---
@pytest.fixture(scope="module")
def big():
    """The 34M-edge workload as the benchmark loads it (degree order)."""
    rp, col = synth.workload("cl_n4m")
    order, nrp, ncol = degree_order(rp, col)
    og = oracle.OracleGraph(nrp, ncol)
    g = moss.Graph(rp, col, order=moss.ORDER_DEGREE)
    yield rp, order, nrp, og, g
    g.close()


def test_large_renumbering(big):
    rp, order, nrp, og, g = big
    n = len(rp) - 1
    assert np.array_equal(moss.moss_table_export(g.handle, moss.TABLE_ORDER, np.zeros(n, dtype=np.uint32)), order)
    vert = moss.moss_table_export(g.handle, moss.TABLE_VERT, np.zeros((n, 4), dtype=np.uint32))
    assert np.array_equal(vert[:, 0], nrp[:-1].astype(np.uint32))
    deg, S, Q, gam = og.vertex()
    assert np.array_equal(vert[:, 2], S.astype(np.uint32))


@pytest.mark.parametrize("method,first", [(0, 123_457), (1, 7), (2, (1 << 26) + 4_099)])
def test_large_slice_counts_match_oracle(big, method, first):
    """Counts of 4e7 ids of each method on the renumbered 34M-edge graph
    (Path-5's slice crosses a 2^26-id deferral chunk) against the oracle's."""
    rp, order, nrp, og, g = big
    count = 40_000_000
    assert np.array_equal(counts(g, method, first, count, 42), oracle_counts(og, method, 42, first, count))


@pytest.mark.parametrize("method", [1, 2])
def test_large_budget_tail_records(big, method):
    """The last 4,000 samples of each sub-method of the benchmark's k = 5,
    1e9-sample step, in input ids."""
    rp, order, nrp, og, g = big
    K = 500_000_000
    cls, verts = records(g, method, K - 4000, 4000, 42)
    _, ocls, overts = og.run(method, 42, 4000, first=K - 4000, record=True)
    assert np.array_equal(cls, ocls)
    assert np.array_equal(verts, order[overts.astype(np.int64)])
