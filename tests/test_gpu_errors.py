"""Invalid inputs are rejected with a status, on the host or by the device
validation pass (whose reads stay inside the copied arrays), and the context
stays usable afterwards."""
from __future__ import annotations

import numpy as np
import pytest

import synth
import paper_1509_08089_gb300 as moss

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def csr(lists):
    rp = np.zeros(len(lists) + 1, dtype=np.uint64)
    for i, l in enumerate(lists):
        rp[i + 1] = rp[i] + len(l)
    col = np.array([x for l in lists for x in l], dtype=np.uint32)
    return rp, col


@pytest.mark.parametrize("lists,word", [
    ([[1], [], [0]], "reverse"),                 # 0->1 and 2->0 without reverses
    ([[2, 1], [0], [0]], "increasing"),          # unsorted list
    ([[0, 1], [0, 1]], "self loop"),             # self loops
    ([[1, 1], [0, 0]], "increasing"),            # duplicate edge
    ([[5], [0]], "n"),                           # id out of range
])
def test_invalid_csr_rejected(lists, word):
    rp, col = csr(lists)
    with pytest.raises(moss.MossError) as ei:
        moss.moss_graph_load_csr(rp, col)
    assert ei.value.status == moss.MOSS_EGRAPH
    assert word in str(ei.value)


def test_bad_row_ptr_rejected():
    rp = np.array([0, 3, 2, 4], dtype=np.uint64)
    col = np.array([1, 2, 0, 0], dtype=np.uint32)
    with pytest.raises(moss.MossError) as ei:
        moss.moss_graph_load_csr(rp, col)
    assert ei.value.status == moss.MOSS_EGRAPH and "row_ptr" in str(ei.value)


def test_state_and_argument_errors():
    rp, col = synth.star(5)
    with moss.Graph(rp, col, k_mask=0) as g:
        with pytest.raises(moss.MossError) as ei:
            moss.moss_sample_estimate(g.handle, 4, 100, 1)
        assert ei.value.status == moss.MOSS_ESTATE
        moss.moss_build_tables(g.handle, 1 << 4)
        with pytest.raises(moss.MossError) as ei:
            moss.moss_sample_estimate(g.handle, 3, 100, 1)
        assert ei.value.status == moss.MOSS_EINVAL
        c = torch.zeros(22, dtype=torch.int64, device="cuda")
        with pytest.raises(moss.MossError) as ei:   # star: Gamma = 0, no sample exists
            moss.moss_sample_counts(g.handle, 0, 0, 10, 1, c)
        assert ei.value.status == moss.MOSS_EINVAL
        with pytest.raises(moss.MossError) as ei:
            moss.moss_build_tables(g.handle, 1 << 3)
        assert ei.value.status == moss.MOSS_EINVAL
        r = g.estimate(4, 100, 1)          # still usable; Gamma = 0 gives n_2 = Lambda_3
        assert r["est"][2] == 10.0 and r["K"] == (0, 0)
    with moss.Graph(rp, col, probe=moss.PROBE_SEARCH) as g:
        moss.moss_set_probe(g.handle, moss.PROBE_HASH)       # hash not built yet
        with pytest.raises(moss.MossError) as ei:
            moss.moss_sample_estimate(g.handle, 5, 100, 1)
        assert ei.value.status == moss.MOSS_ESTATE
        with pytest.raises(moss.MossError) as ei:
            moss.moss_set_probe(g.handle, 7)
        assert ei.value.status == moss.MOSS_EINVAL
    with moss.Graph(rp, col, probe=moss.PROBE_HASH) as g:
        moss.moss_set_probe(g.handle, moss.PROBE_FILTER)     # filter not built yet
        with pytest.raises(moss.MossError) as ei:
            moss.moss_sample_estimate(g.handle, 4, 100, 1)
        assert ei.value.status == moss.MOSS_ESTATE
    with pytest.raises(moss.MossError) as ei:
        moss.moss_graph_load_csr(rp, col, device=99)
    assert ei.value.status == moss.MOSS_EINVAL
    # after all of the above the device still works
    rp, col = synth.cycle(8)
    with moss.Graph(rp, col) as g:
        assert g.estimate(4, 1000, 2)["est"][1] == pytest.approx(8.0)


def test_gather_rate():
    # the measurement helper: L2-resident random sector reads are served
    # faster than ones spread over a buffer far larger than L2
    l2 = moss.moss_gather_rate(64 << 20)
    hbm = moss.moss_gather_rate(2 << 30)
    assert l2 > 0 and hbm > 0
    assert l2 > 2 * hbm
    with pytest.raises(moss.MossError) as ei:
        moss.moss_gather_rate(48)
    assert ei.value.status == moss.MOSS_EINVAL
