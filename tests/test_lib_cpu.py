"""The C ABI library without a GPU: it loads, exports every function the
header declares, and rejects bad arguments before touching the device."""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np
import pytest

import paper_1509_08089_gb300 as moss
from conftest import ROOT, gpu_available

HEADER = os.path.join(ROOT, "include", "moss.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(moss_[a-z_0-9]+)\s*\(", src)))


def test_library_exports_every_declared_function():
    from paper_1509_08089_gb300 import build
    build.build()
    lib = ctypes.CDLL(moss.LIB_PATH)
    names = declared_functions()
    assert len(names) >= 12
    for name in names:
        assert hasattr(lib, name), name


def test_binding_covers_every_declared_function():
    for name in declared_functions():
        assert hasattr(moss, name), name


def test_strings():
    assert moss.moss_version().startswith("moss-gb300")
    assert moss.moss_strerror(moss.MOSS_EGRAPH) == "invalid graph"
    assert moss.moss_strerror(12345) == "unknown status"


def test_argument_checks_before_device():
    lib = moss.load()
    out = ctypes.c_void_p()
    rp = np.array([0, 1, 2], dtype=np.uint64)
    col = np.array([1, 0], dtype=np.uint32)
    assert lib.moss_graph_load_csr(rp.ctypes.data, 1, col.ctypes.data, 2, 2, 0, None, None) == moss.MOSS_EINVAL
    assert lib.moss_graph_load_csr(None, 1, col.ctypes.data, 2, 2, 0, None, ctypes.byref(out)) == moss.MOSS_EINVAL
    assert lib.moss_graph_load_csr(rp.ctypes.data, 1, col.ctypes.data, 0, 2, 0, None, ctypes.byref(out)) == moss.MOSS_EINVAL
    assert lib.moss_graph_load_csr(rp.ctypes.data, 1, col.ctypes.data, 2, 1 << 32, 0, None,
                                   ctypes.byref(out)) == moss.MOSS_EOVERFLOW
    assert lib.moss_graph_load_csr(rp.ctypes.data, 1, col.ctypes.data, 2, 3, 0, None,
                                   ctypes.byref(out)) == moss.MOSS_EGRAPH
    assert b"odd" in lib.moss_last_error_detail()
    assert lib.moss_graph_load_csr_order(rp.ctypes.data, 1, col.ctypes.data, 2, 2, 2, 0, None,
                                         ctypes.byref(out)) == moss.MOSS_EINVAL
    r = moss.moss_result()
    assert lib.moss_sample_estimate(None, 4, 10, 1, None, ctypes.byref(r)) == moss.MOSS_EINVAL
    assert lib.moss_build_tables(None, 16, None) == moss.MOSS_EINVAL
    assert lib.moss_sample_counts(None, 0, 0, 1, 1, None, None) == moss.MOSS_EINVAL
    assert lib.moss_sample_estimate_min(None, 10, 10, 1, None, ctypes.byref(r)) == moss.MOSS_EINVAL
    K = np.zeros(2, dtype=np.uint64)
    H = np.zeros(44, dtype=np.uint64)
    assert lib.moss_finalize_min(None, K.ctypes.data, H.ctypes.data, None, None, ctypes.byref(r)) == moss.MOSS_EINVAL
    rate = ctypes.c_double(1.0)
    assert lib.moss_gather_rate(64 << 20, 0, None, None) == moss.MOSS_EINVAL
    assert lib.moss_gather_rate(0, 0, None, ctypes.byref(rate)) == moss.MOSS_EINVAL and rate.value == 0.0
    assert lib.moss_gather_rate(33, 0, None, ctypes.byref(rate)) == moss.MOSS_EINVAL
    assert lib.moss_gather_rate(64 << 20, -1, None, ctypes.byref(rate)) == moss.MOSS_EINVAL
    lib.moss_graph_free(None)


@pytest.mark.skipif(gpu_available(), reason="checks the no-GPU failure path")
def test_fails_loudly_without_gpu():
    rp = np.array([0, 1, 2], dtype=np.uint64)
    col = np.array([1, 0], dtype=np.uint32)
    with pytest.raises(moss.MossError) as ei:
        moss.moss_graph_load_csr(rp, col)
    assert ei.value.status in (moss.MOSS_ECUDA, moss.MOSS_EINVAL)


def test_result_struct_layout_matches_header():
    # doubles after uint64 arrays: no padding surprises between C and ctypes
    assert ctypes.sizeof(moss.moss_result) == 4 + 4 + 16 + 2 * 22 * 8 + 22 * 8 * 2 + 2 * 22 * 8 + 16 + 22 * 8
    assert ctypes.sizeof(moss.moss_stats) == 8 + 8 + 8 + 64 + 16 + 16 + 32 + 16
