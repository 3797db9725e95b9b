"""moss_sample_counts_noalloc against moss_sample_counts.

The no-allocation entry point exists for callers that may not allocate
device memory while they run (a fixed memory budget reserved at start-up, a
loop that cannot take an allocation's device synchronisation, an allocator
owned by another framework).  It keeps the sampler's per-block partial counts
in one fixed array inside the library.  Its counts must equal the ordinary
entry point's exactly (integer counts), on two calls in a row -- the array
keeps the previous call's contents, so the second call, with a different
range and method, would expose stale rows.  This file is collected last so
that a run stopping at the first failure has run every other test.
"""
from __future__ import annotations

import numpy as np
import pytest

import synth
import paper_1509_08089_gb300 as moss

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def counts(fn, g, method, first, count, seed):
    out = torch.full((22,), -1, dtype=torch.int64, device="cuda")
    fn(g.handle, method, first, count, seed, out)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def test_noalloc_counts_equal_allocating_counts_twice_in_a_row():
    rp, col = synth.workload("cl_n2k")
    with moss.Graph(rp, col) as g:
        calls = [(2, 1_000, 300_007, 11), (1, 77, 123_451, 12), (0, 5, 99_999, 13)]
        for method, first, count, seed in calls:        # consecutive calls share the array
            ref = counts(moss.moss_sample_counts, g, method, first, count, seed)
            got = counts(moss.moss_sample_counts_noalloc, g, method, first, count, seed)
            assert np.array_equal(got, ref), (method, got, ref)
            assert int(got.sum()) == count
        # the same call twice in a row gives the same counts
        a = counts(moss.moss_sample_counts_noalloc, g, 2, 0, 200_003, 3)
        b = counts(moss.moss_sample_counts_noalloc, g, 2, 0, 200_003, 3)
        assert np.array_equal(a, b)
        assert np.array_equal(a, counts(moss.moss_sample_counts, g, 2, 0, 200_003, 3))


def test_noalloc_rejects_unbuilt_tables():
    rp, col = synth.workload("cl_n2k")
    with moss.Graph(rp, col, k_mask=0) as g:
        out = torch.zeros(22, dtype=torch.int64, device="cuda")
        with pytest.raises(moss.MossError) as ei:
            moss.moss_sample_counts_noalloc(g.handle, 0, 0, 10, 1, out)
        assert ei.value.status == moss.MOSS_ESTATE


def test_noalloc_rejects_missing_probe_tables():
    """Like moss_sample_counts, the no-allocation call refuses a graph whose
    probe strategy names tables that were never built."""
    rp, col = synth.workload("cl_n2k")
    out = torch.zeros(22, dtype=torch.int64, device="cuda")
    with moss.Graph(rp, col, probe=moss.PROBE_SEARCH) as g:
        moss.moss_set_probe(g.handle, moss.PROBE_HASH)        # hashed edge set not built
        for fn in (moss.moss_sample_counts, moss.moss_sample_counts_noalloc):
            with pytest.raises(moss.MossError) as ei:
                fn(g.handle, 1, 0, 1000, 1, out)
            assert ei.value.status == moss.MOSS_ESTATE
    with moss.Graph(rp, col, probe=moss.PROBE_HASH) as g:
        moss.moss_set_probe(g.handle, moss.PROBE_FILTER)      # edge filter not built
        with pytest.raises(moss.MossError) as ei:
            moss.moss_sample_counts_noalloc(g.handle, 0, 0, 1000, 1, out)
        assert ei.value.status == moss.MOSS_ESTATE
