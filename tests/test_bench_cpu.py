"""bench.py's output contract and launch arithmetic, on the CPU: the
reference arm (the CPU oracle) prints one JSON line with the keys the
measurement contract names, and the launch count it claims for the GPU arm
follows the kernels a step runs."""
from __future__ import annotations

import json
import os
import subprocess
import sys

import pytest

from conftest import ROOT

sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_reference_arm_json_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "1", "--workload", "cl_n2k", "--budget", "200000"],
                       capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["value"] > 0 and d["unit"] == "samples/s" and d["higher_is_better"] is True
    assert d["steps"] == 1 and d["warmup"] == 1 and d["n_gpus"] == 1
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": "samples/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert "workload" in d["config"]
    # the GPU line's config keys, with the order --vertex-order auto resolves to (an L2-sized graph: input ids)
    assert d["config"]["vertex_order"] == "input" and d["config"]["probe"] == "hash"


@pytest.mark.parametrize("k,budget,mix,filtered,two,expected", [
    # load 8 + build 8 + finalize 1; T-5: sampler + reduce; Path-5: main, two redraw stages, reduce per chunk
    (5, 100_000_000, False, False, False, 17 + 2 + 4),
    # the edge filter and its 6 hub kernels, two-level vertex tables 3 split
    # kernels; 5e8 Path-5 ids: 8 chunks of 2^26
    (5, 1_000_000_000, False, True, True, 17 + 7 + 3 + 2 + 4 * 8),
    (4, 100_000_000, False, False, False, 17 + 2),
    (4, 100_000_000, True, False, False, 17 + 12 + 2 + 2),    # MOSS-4 + MOSS-4Min with its 12 table kernels
    (4, 100_000_000, True, False, True, 17 + 3 + 15 + 2 + 2),
])
def test_launches_per_step(k, budget, mix, filtered, two, expected):
    assert bench.DEFER_CHUNK == 1 << 26
    assert bench.launches_per_step(k, budget, mix, filtered, two) == expected


def test_launches_follow_the_default_splits():
    # 1M-edge graph (n = 100,000): two-level vertex tables, one-level MOSS-4Min table
    assert bench.default_vertex_splits(100_000) == (12, 64)
    assert bench.default_vertex_splits(4_000_000) == (20, 20)
    assert bench.default_vertex_splits(2_000) == (64, 64)
    assert bench.launches_per_step(4, 100_000_000, True, False, True, False) == 17 + 3 + 12 + 2 + 2
    args = type("A", (), {"vertex_split": -1})()
    assert bench.two_levels(args, 100_000) == (True, False)
    args.vertex_split = 64
    assert bench.two_levels(args, 100_000) == (False, False)


def test_resolved_probe_follows_the_hash_size():
    import numpy as np
    small = np.array([0, 1_000_000], dtype=np.int64)     # 2^19 buckets of 32 B: 16 MiB
    large = np.array([0, 68_000_000], dtype=np.int64)    # 2^26 buckets: 2 GiB
    assert bench.resolved_probe("auto", small) == "hash"
    assert bench.resolved_probe("auto", large) == "filter"
    assert bench.resolved_probe("search", large) == "search"


def test_default_splits_match_the_oracle():
    import oracle
    for n in (100, (1 << 14) - 1, 1 << 14, 100_000, (1 << 20) - 1, 1 << 20, 4_000_000):
        assert bench.default_vertex_splits(n) == (oracle.default_split(n), oracle.default_split_min(n)), n


def test_vertex_order_follows_the_table_size():
    """auto: degree order exactly when the sampling tables exceed the L2."""
    import numpy as np
    l2 = bench.GB300_L2_BYTES
    small = np.zeros(100_001, dtype=np.uint64)
    small[-1] = 2_000_000
    large = np.zeros(4_000_001, dtype=np.uint64)
    large[-1] = 68_000_000
    assert bench.resolved_order("auto", small, "hash", [1, 2], l2) == "input"
    assert bench.resolved_order("auto", large, "filter", [1, 2], l2) == "degree"
    assert bench.resolved_order("input", large, "filter", [1, 2], l2) == "input"
    assert bench.resolved_order("degree", small, "hash", [1, 2], l2) == "degree"
    assert bench.data_key("cl_n4m", "degree") == "cl_n4m_degree" and bench.data_key("cl_n4m", "input") == "cl_n4m"
    # four more kernels per step in degree order: key counts, their scan, placement, lists
    base = bench.launches_per_step(5, 1_000_000_000, False, True, True)
    assert bench.launches_per_step(5, 1_000_000_000, False, True, True, ordered=True) == base + 4


@pytest.mark.parametrize("key,traffic_keys,resident", [
    ("cl_n100k", ["MOSS4_hash", "T5_hash", "PATH5_hash", "MOSS4MIN_hash"], True),
    ("cl_n4m", ["MOSS4_filter", "T5_filter", "PATH5_filter"], False),
    ("cl_n4m_degree", ["MOSS4_filter", "T5_filter", "PATH5_filter"], False),
])
def test_roofline_data_files(key, traffic_keys, resident):
    """The sector figures and DRAM captures the roofline reads for each
    workload and vertex order: every figure present; while the captures
    match the sampler source, each fitted traffic per sample positive and
    below the algorithmic bytes on the L2-resident graph (the L2 serves
    most reads), within a factor of four of them on the HBM-resident one."""
    import json
    sect = json.load(open(os.path.join(ROOT, "tests", "golden", f"sectors_{key}.json")))
    for k in traffic_keys:
        spb = sect[k]["sectors_per_sample"]
        assert 4.0 < spb < 40.0, (key, k)
    fits = {k: bench.small_case_traffic(key, k, 500_000_000) for k in traffic_keys}
    if any(tb is None for tb, _ in fits.values()):
        pytest.skip("DRAM captures predate the current sampler source (traffic reported as null)")
    for k, (tb, how) in fits.items():
        per = tb / 500_000_000
        alg = sect[k]["sectors_per_sample"] * 32.0
        if resident:
            assert 0 < per < alg, (key, k, per, alg)
        else:
            assert alg / 4 < per < 4 * alg, (key, k, per, alg)
        assert "samples" in how
