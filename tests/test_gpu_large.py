"""The maximum-size workload: Chung-Lu n=4M, exponent 2.1, mean degree 17,
max degree 20,000 (~35M edges, ~1.4 GB of device tables), 1e9 samples per
motif size.  Tables are compared with the oracle's bit for bit, samples one
by one at the end of the 1e9 range, the full-budget counts by their
invariants and by the finalize of the same counts, and the counts of a
1.4e8-id slice of every method with the oracle's over the same ids (Path-5's
slice starts past the first 2^26-id deferral chunk and spans three of them)."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import synth
import paper_1509_08089_gb300 as moss
from helpers import expected_slot_neighbour, oracle_counts, slot_twin
from oracle.finalize import PHI5

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def big():
    rp, col = synth.workload("cl_n4m")
    og = oracle.OracleGraph(rp, col)
    g = moss.Graph(rp, col)
    yield rp, col, og, g
    g.close()


def test_large_tables_bit_exact(big):
    rp, col, og, g = big
    n, nnz = og.n, og.nnz
    deg, S, Q, gam = og.vertex()
    vert = moss.moss_table_export(g.handle, moss.TABLE_VERT, np.zeros((n, 4), dtype=np.uint32))
    assert np.array_equal(vert[:, 1], deg.astype(np.uint32))
    assert np.array_equal(vert[:, 2], S.astype(np.uint32))
    thr, alias, acc = og.sigma_table()
    slot = moss.moss_table_export(g.handle, moss.TABLE_SLOT, np.zeros((nnz, 8), dtype=np.uint32))
    assert np.array_equal(slot[:, 2], thr.astype(np.uint32))
    assert np.array_equal(slot[:, 3], alias)
    owner = np.repeat(np.arange(n, dtype=np.int64), deg.astype(np.int64))
    twin = slot_twin(slot)
    assert np.array_equal(col[rp.astype(np.int64)[col.astype(np.int64)] + twin], owner)
    nb, off = expected_slot_neighbour(rp, col, twin)
    assert np.array_equal(slot[:, 1], nb)
    assert np.array_equal(slot[:, 4], off)
    apos = rp.astype(np.int64)[owner] + slot[:, 3].astype(np.int64)
    assert np.array_equal(slot[:, 5:8], slot[apos][:, [0, 1, 4]])
    for l in range(3):
        vt = og.vertex_table(l)
        assert moss.moss_vertex_levels(g.handle, l) == (vt["nh"], vt["TL"]), l
        assert 0 < vt["nh"] < 100_000 and vt["TL"] > 0, l     # both levels hold weight
        seed = moss.moss_table_export(g.handle, moss.TABLE_SEED0 + l, np.zeros((n, 8), dtype=np.uint32))
        Tg = seed[:, 0].astype(np.uint64) | (seed[:, 1].astype(np.uint64) << np.uint64(32))
        assert np.array_equal(Tg, vt["T"]), l
        assert np.array_equal(seed[:, 2], vt["alias"]), l
        assert np.array_equal(seed[:, 3], vt["self"]), l
        assert np.array_equal(seed[:, 4:8], vert[vt["alias"].astype(np.int64)]), l
    st = g.stats()
    for l in range(3):
        assert (int(st.gamma[l][0]) | (int(st.gamma[l][1]) << 64)) == og.Gamma[l]


@pytest.mark.parametrize("k", [4, 5])
def test_large_full_budget(big, k):
    rp, col, og, g = big
    B = 1_000_000_000
    r = g.estimate(k, B, seed=42)
    if k == 4:
        assert tuple(r["K"]) == (B, 0) and int(r["hits"][0].sum()) == B
        o = oracle.finalize_moss4(r["hits"][0], B, og.Gamma[0], og.Lambda3)
        methods = [(0, B)]
    else:
        K1, K2 = B // 2, B - B // 2
        assert tuple(r["K"]) == (K1, K2)
        assert int(r["hits"][0].sum()) == K1 and int(r["hits"][1].sum()) == K2
        for i in range(1, 22):
            if PHI5[i - 1, 0] == 0:
                assert r["hits"][0][i] == 0
            if PHI5[i - 1, 1] == 0:
                assert r["hits"][1][i] == 0
        o = oracle.finalize_moss5(r["hits"][0], r["hits"][1], K1, K2, og.Gamma[1], og.Gamma[2], og.Lambda4)
        methods = [(1, K1), (2, K2)]
    n = 7 if k == 4 else 22
    lam = float(og.Lambda3 if k == 4 else og.Lambda4)
    for i in range(1, n):
        tol = 1e-9 * (max(lam, 1.0) if i == 2 else max(abs(o["est"][i]), 1e-300))
        assert abs(r["est"][i] - o["est"][i]) <= tol, (k, i)
    for method, K in methods:
        cls = torch.empty(4000, dtype=torch.uint8, device="cuda")
        verts = torch.empty(4000 * 5, dtype=torch.int32, device="cuda")
        moss.moss_sample_records(g.handle, method, K - 4000, 4000, 42, cls, verts)
        torch.cuda.synchronize()
        _, ocls, overts = og.run(method, 42, 4000, first=K - 4000, record=True)
        assert np.array_equal(cls.cpu().numpy(), ocls)
        ncol = 4 if method == 0 else 5
        assert np.array_equal(verts.cpu().numpy().view(np.uint32).reshape(4000, 5)[:, :ncol], overts[:, :ncol])


SLICE = 140_000_000


@pytest.mark.parametrize("method,first", [(0, 123_457), (1, 7), (2, (1 << 26) + 4_099)])
def test_large_slice_counts_match_oracle(big, method, first):
    """The counts of ids [first, first + 1.4e8) of one method, drawn by the
    library's sampling call, equal the oracle's over the same ids."""
    rp, col, og, g = big
    counts = torch.zeros(22, dtype=torch.int64, device="cuda")
    moss.moss_sample_counts(g.handle, method, first, SLICE, 42, counts)
    torch.cuda.synchronize()
    got = counts.cpu().numpy().view(np.uint64)
    assert int(got.sum()) == SLICE
    assert np.array_equal(got, oracle_counts(og, method, 42, first, SLICE))
