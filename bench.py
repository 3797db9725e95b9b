#!/usr/bin/env python
"""Benchmark of the whole sampling path on one GPU per rank.

A step is one pass of the path over the 1M-edge workload: load the CSR
(already in HBM) and validate it with the vertex weights (a0), build the
alias tables (a1), draw and classify the samples and count them (a2-a8),
finalize the estimates (a9), free the graph.  Default workload: Chung-Lu
n = 100,000, exponent 2.2, mean degree 20, max degree 5,000, seed 1 (~1M
edges), k = 5 (T-5 + Path-5), budget 1e8 samples per rank (weak scaling).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Prints one JSON line (rank 0).  On one GPU the line also carries, each with
its own clock record, the other terms of the headline measurement:
``config3`` (the same step on the 34M-edge Chung-Lu graph, 1e9 samples,
against the HBM roofline), ``batched`` (512 uneven graphs in one persistent
launch against one launch per request) and ``served`` (a Poisson request
stream with target errors against one request per launch).  --impl reference
times the CPU oracle on a bounded sample of the same workload instead (rank 0
only).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

GRAPHS = {
    "cl_n2k": ("Chung-Lu n=2,000, exponent 2.5, mean degree 8, max degree 200, seed 1 (7,886 edges)", "8k edges"),
    "cl_n100k": ("Chung-Lu n=100,000, exponent 2.2, mean degree 20, max degree 5,000, seed 1 (~1M edges)",
                 "1M edges"),
    "cl_n4m": ("Chung-Lu n=4,000,000, exponent 2.1, mean degree 17, max degree 20,000, seed 1 (~34M edges)",
               "34M edges"),
}


def describe(workload: str, k: int, mix: bool = False) -> tuple[str, str]:
    """(metric, workload description) of a run."""
    graph, size = GRAPHS[workload]
    if mix:
        return (f"4-node samples/s at {size} (MOSS-4 + MOSS-4Min)",
                f"{graph}, k=4 MOSS-4 and MOSS-4Min with K = K-check, sorted uint32 CSR")
    method = "k=5 (T-5 + Path-5, K1=K2)" if k == 5 else "k=4 (MOSS-4)"
    return f"{k}-node samples/s at {size}", f"{graph}, {method}, sorted uint32 CSR"


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    p.add_argument("--workload", default="cl_n100k")
    p.add_argument("--k", type=int, default=5)
    p.add_argument("--budget", type=int, default=100_000_000)
    p.add_argument("--seed", type=int, default=42)
    p.add_argument("--e2e-steps", type=int, default=3)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--mode", default="single", choices=["single", "batch", "serve", "min", "call"],
                   help="single: the one-graph step; batch: many graphs in one persistent launch; serve: "
                        "the request server; min: the one-graph step of MOSS-4 + MOSS-4Min (k=4); call: "
                        "sampling calls of given methods and sizes alone (for profiler captures)")
    p.add_argument("--methods", default="1,2", help="call mode: methods (0 MOSS-4, 1 T-5, 2 Path-5, 3 MOSS-4Min)")
    p.add_argument("--counts", default="5000000,10000000", help="call mode: samples per call")
    p.add_argument("--graphs", type=int, default=512, help="batch mode: number of graphs")
    p.add_argument("--rate", type=float, default=2000.0, help="serve mode: mean arrivals per second")
    p.add_argument("--duration", type=float, default=2.0, help="serve mode: seconds of arrivals")
    p.add_argument("--no-extras", action="store_true",
                   help="single mode: leave out the 34M-edge, batched and served terms of the line")
    p.add_argument("--serve-duration", type=float, default=1.0,
                   help="seconds of Poisson arrivals of the served term of the default line")
    p.add_argument("--rng", default="splitmix64", choices=["splitmix64", "philox4x32"],
                   help="word generator of the samples (both sides of the comparison use it)")
    p.add_argument("--vertex-split", type=int, default=-1,
                   help="vertex-table level split of the workload's graph (0..64; default: the library's)")
    p.add_argument("--vertex-order", default="auto", choices=["auto", "input", "degree"],
                   help="internal vertex order of the loads: auto (degree order when the sampling tables "
                        "exceed the L2, else the input ids), the input ids, or degree order")
    p.add_argument("--probe", default="auto", choices=["auto", "hash", "filter", "search"],
                   help="induced-edge tests: auto (filtered set when the set exceeds 64 MiB, else the set), "
                        "hashed edge set, set behind a Bloom filter, or sorted-list search")
    return p.parse_args()


# ----------------------------------------------------------- CPU (oracle) --
def _oracle_worker(args):
    """One process of the CPU baseline: build the oracle's tables for the
    workload, then draw its share of samples of each sub-method."""
    workload, k, seed, shares, rng, vsplit = args
    sys.path.insert(0, ROOT)
    import oracle
    import synth
    rp, col = synth.workload(workload)
    t0 = time.perf_counter()
    g = oracle.OracleGraph(rp, col, vsplit=vsplit)
    if any(m == oracle.MOSS4MIN for m, _, _ in shares):
        g.build_min()
    t1 = time.perf_counter()
    for method, first, count in shares:
        g.run(method, seed, count, first=first, rng=rng)
    t2 = time.perf_counter()
    return t1 - t0, t2 - t1, sum(c for _, _, c in shares)


def sub_methods(k, mix=False):
    return ([0, 3] if mix else [0]) if k == 4 else [1, 2]


def oracle_pass(pool, cores, workload, k, seed, per_worker, mix=False, rng=0, vsplit=None):
    methods = sub_methods(k, mix)
    jobs = []
    for w in range(cores):
        shares = [(m, w * per_worker // len(methods), per_worker // len(methods)) for m in methods]
        jobs.append((workload, k, seed, shares, rng, vsplit))
    t0 = time.perf_counter()
    res = list(pool.map(_oracle_worker, jobs))
    wall = time.perf_counter() - t0
    build = max(r[0] for r in res)
    sample_wall = max(r[1] for r in res)
    samples = sum(r[2] for r in res)
    return build, sample_wall, samples, wall


def oracle_rate(build, sample_wall, samples, budget):
    """Whole-path throughput of the oracle extrapolated to the full budget:
    one table build plus budget samples at the measured sampling rate."""
    rate = samples / sample_wall
    return budget / (build + budget / rate), rate


def bench_config(args, rp, world: int, workload: str | None = None, order: str = "input") -> dict:
    """The `config` object of a line; both arms print the same one."""
    wl = workload or describe(args.workload, args.k, args.mode == "min")[1]
    cfg = {"workload": wl, "budget_per_gpu": args.budget, "seed": args.seed,
           "probe": resolved_probe(args.probe, rp), "rng": args.rng, "vertex_order": order,
           "l2": "GPU arm: flushed (512 MB write) before every timed step; CPU oracle: not applicable",
           "parallelism": f"replicas x{world}"}
    if args.vertex_split >= 0:
        cfg["vertex_split"] = args.vertex_split
    return cfg


RNG_IDS = {"splitmix64": 0, "philox4x32": 1}   # the same numbering on both sides


def calibrate_per_worker(workload, k, seed, seconds, mix=False, rng=0, vsplit=None):
    """Samples per worker process for about `seconds` of sampling, and the
    oracle's sampling rate on one core (samples/s) measured on the way."""
    import oracle
    import synth
    rp, col = synth.workload(workload)
    g = oracle.OracleGraph(rp, col, vsplit=vsplit)
    methods = sub_methods(k, mix)
    if mix:
        g.build_min()
    n = 20_000
    t0 = time.perf_counter()
    for m in methods:
        g.run(m, seed, n // len(methods), rng=rng)
    per = (time.perf_counter() - t0) / n
    return max(len(methods), int(seconds / per)), 1.0 / per


def make_pool(cores):
    import concurrent.futures as cf
    import multiprocessing as mp
    return cf.ProcessPoolExecutor(max_workers=cores, mp_context=mp.get_context("spawn"))


def run_reference(args):
    """The oracle timed on all host cores.  A step is a bounded sample of the
    workload: every core's process builds the oracle's tables of the graph
    and draws its share of per_worker samples (sub-methods split evenly), about
    four seconds in all; value = samples drawn / the step's wall time, both as
    measured (no extrapolation)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import synth
    mix = args.mode == "min"
    if mix:
        args.k = 4
    METRIC, _ = describe(args.workload, args.k, mix)
    rp, _col = synth.workload(args.workload)
    cores = os.cpu_count() or 1
    rng = RNG_IDS[args.rng]
    vsplit = args.vertex_split if args.vertex_split >= 0 else None
    per_worker, single = calibrate_per_worker(args.workload, args.k, args.seed, 4.0, mix, rng, vsplit)
    with make_pool(cores) as pool:
        for _ in range(args.warmup):
            oracle_pass(pool, cores, args.workload, args.k, args.seed, per_worker, mix, rng, vsplit)
        walls, counts = [], []
        for _ in range(args.steps):
            b, sw, n, wall = oracle_pass(pool, cores, args.workload, args.k, args.seed, per_worker, mix, rng, vsplit)
            walls.append(wall)
            counts.append(n)
    samples = counts[0]
    wall = statistics.median(walls)
    v = samples / wall
    split = "T-5/Path-5" if args.k == 5 else ("MOSS-4/MOSS-4Min" if mix else "MOSS-4")
    order = resolved_order(args.vertex_order, rp, resolved_probe(args.probe, rp), sub_methods(args.k, mix),
                           GB300_L2_BYTES)
    sample = (f"{samples} of the workload's {args.budget} samples per step ({split} split evenly) over {cores} "
              f"processes, each building the oracle's tables of the graph (input ids); value = samples / "
              f"measured step time")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": "samples/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * wall, "samples_per_step": samples,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
        "config": bench_config(args, rp, args.gpus, order=order),
        "cpu_baseline": {"value": v, "unit": "samples/s", "cores": cores, "kind": "oracle", "sample": sample,
                         "single_core_sampling_rate": single},
        "e2e": {"value": v, "unit": "samples/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "step_ms": [1000 * w for w in walls],
    }), flush=True)


# ---------------------------------------------------------------- clocks --
class Clocks:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        # the raw samples go to MOSS_CLOCKS_DIR when set (kept for inspection),
        # else to a per-process temporary file; the JSON line carries the summary
        d = os.environ.get("MOSS_CLOCKS_DIR")
        self.path = (os.path.join(d, f"clocks_rank{device}.csv") if d and os.path.isdir(d)
                     else os.path.join(tempfile.gettempdir(), f"moss_clocks_{os.getpid()}_{device}.csv"))

    def start(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "50"], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
            return
        # the sampler's start-up (driver and NVML initialisation) stalls the
        # host for milliseconds: let it finish before the timed region
        t0 = time.perf_counter()
        while time.perf_counter() - t0 < 5.0 and self.proc.poll() is None:
            self.f.flush()
            if os.path.getsize(self.path) > 0:
                break
            time.sleep(0.01)

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------------- GPU --
DEFER_CHUNK = 1 << 26   # Path-5 sample ids per main/deferred launch pair


def resolved_probe(name: str, row_ptr) -> str:
    """The strategy the library picks for --probe auto: the filtered set when
    the hashed set (next power of two >= nnz / 2 buckets of 32 B) exceeds
    64 MiB."""
    if name != "auto":
        return name
    nnz, b = int(row_ptr[-1]), 2
    while b < (nnz + 1) // 2:
        b <<= 1
    return "filter" if b * 32 > (64 << 20) else "hash"


def resolved_order(name: str, row_ptr, probe: str, methods, l2_bytes: int) -> str:
    """The vertex order --vertex-order auto picks: the graph loaded in degree
    order when the tables a sampling call reads exceed the L2 (their records
    then come from HBM, and grouping the heavy vertices puts the hot ones in
    fewer lines), else the input ids (an L2-resident graph gains nothing
    that pays for the renumbering)."""
    if name != "auto":
        return name
    return "degree" if sampler_tables_bytes(row_ptr, probe, methods) > l2_bytes else "input"


ORDER_IDS = {"input": 0, "degree": 1}
GB300_L2_BYTES = 135_528_448   # the device's L2 (cudaDevAttrL2CacheSize); the CPU arm has no device to ask


def data_key(workload: str, order: str) -> str:
    """Name of a workload's sector-model and DRAM-capture files: the degree
    order has its own (the layout of the renumbered graph)."""
    return workload + ("_degree" if order == "degree" else "")


def default_vertex_splits(n: int) -> tuple[int, int]:
    """The library's default level splits of a graph of n vertices: of the
    vertex tables of Gamma, Gamma^(1), Gamma^(2), and of the MOSS-4Min
    table (64: one level)."""
    if n >= 1 << 20:
        return 20, 20
    return (12, 64) if n >= 1 << 14 else (64, 64)


def two_levels(args, n: int) -> tuple[bool, bool]:
    """Whether the build splits the vertex tables (and the MOSS-4Min table)
    into two levels under the run's vertex split."""
    if args.vertex_split >= 0:
        return args.vertex_split < 64, args.vertex_split < 64
    main, mn = default_vertex_splits(n)
    return main < 64, mn < 64


def launches_per_step(k: int, budget: int, mix: bool, filtered: bool = False, two_level: bool = False,
                      two_level_min: bool | None = None, ordered: bool = False) -> int:
    """Kernels of one step: load 8 (vertices, owners, slot weights, short and
    long slot scans, twins, vertex weights, totals), 4 more in degree order
    (key counts, their scan, the placement, the lists); build 8 (two sigma alias passes, the
    alias-half fill, four alias phases of the vertex tables, edge hash), 3
    more (the level split) for two-level vertex tables, 7 more behind the
    edge filter (the filter, and the hubs' degree histogram, degree cut,
    rank-table bits, their scan, the prefixes and list, and the adjacency
    bits); MOSS-4Min build 12
    (three sort tiers, slot records, two alias passes, pick records, total,
    four alias phases of its vertex table), again 3 more with two levels; per
    sub-method a sampler and a reduce, Path-5 per chunk of DEFER_CHUNK ids a
    main launch, the second-attempt and fallback launches and a reduce; one
    finalize."""
    from paper_1509_08089_gb300.dist import sub_budgets
    split = 3 if two_level else 0
    split_min = split if two_level_min is None else (3 if two_level_min else 0)
    n = 8 + (4 if ordered else 0) + 8 + split + (7 if filtered else 0) + ((12 + split_min) if mix else 0) + 1
    for m, K in sub_budgets(k, budget, mix):
        n += 4 * -(-K // DEFER_CHUNK) if m == 2 else 2
    return n


def peaks_file() -> dict:
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    return json.load(open(path)) if os.path.exists(path) else {}


def sampler_tables_bytes(rp, probe: str, methods) -> int:
    """Bytes of the device tables a sampling call reads, by the library's
    layout: 32 B slot records and 4 B ids per list entry, 16 B vertex records
    and a 32 B vertex alias record per vertex and method, and the hashed edge
    set (32 B buckets, the next power of two >= nnz / 2) or the edge filter in
    front of it (4 B words, the largest power of two <= nnz / 8) with the
    hubs' rank table (8 B per 32 vertices) and adjacency bits (H^2,
    H = min(8192, max(16, n / 16)))."""
    n, nnz = len(rp) - 1, int(rp[-1])
    total = nnz * (32 + 4) + n * (16 + 32 * len(methods))
    if probe in ("hash", "filter"):
        b = 2
        while b < (nnz + 1) // 2:
            b <<= 1
        total += 32 * b
    if probe == "filter":
        w = 1
        while 2 * w <= max(nnz // 8, 1):
            w <<= 1
        total += 4 * w
        h = min(8192, max(16, n // 16))
        total += 8 * ((n + 31) // 32) + (h * h + 31) // 32 * 4
    return total


def small_case_traffic(workload: str, key: str, samples: int):
    """DRAM bytes (read + write) of one sampling call of `samples` ids,
    scaled from the small-case ncu captures in
    profiles/dram_traffic_small_<workload>.txt: with captures at two or more
    sizes the bytes are fitted as a + b * samples (a: the cold start of the
    tables), with one capture scaled in proportion.  None when the file is
    missing or the sampler source changed since the capture."""
    import hashlib
    path = os.path.join(ROOT, "profiles", f"dram_traffic_small_{workload}.txt")
    if not os.path.exists(path):
        return None, None
    rec, pts = {}, []
    for line in open(path):
        if not line.strip() or line.startswith("#"):
            continue
        a, b = line.split()[:2]
        if "@" in a:
            k, n = a.split("@")
            if k == key:
                pts.append((float(n), float(b)))
        else:
            rec[a] = b
    src = b"".join(open(os.path.join(ROOT, "paper_1509_08089_gb300", "csrc", f), "rb").read()
                   for f in ("moss_sample.cu", "moss_internal.cuh"))
    if hashlib.sha256(src).hexdigest()[:16] != rec.get("source_sha") or not pts:
        return None, None
    if len(pts) == 1:
        return pts[0][1] * samples / pts[0][0], f"one capture of {int(pts[0][0])} samples, scaled in proportion"
    x = np.array([q[0] for q in pts])
    y = np.array([q[1] for q in pts])
    b1, a0 = np.polyfit(x, y, 1)
    sizes = "/".join(str(int(q)) for q in x)
    return float(a0 + b1 * samples), f"fit a + b*samples over captures of {sizes} samples"


def time_calls(moss, torch, h, k, budget, mix, seed, stream, l2_flush, reps=3):
    """CUDA-event time of each sub-method's sampling call alone (the calls
    the step makes), after one untimed call, L2 flushed before each."""
    from paper_1509_08089_gb300.dist import sub_budgets
    counts = torch.zeros(22, dtype=torch.int64, device=l2_flush.device)
    times = {}
    for m, K in sub_budgets(k, budget, mix):
        moss.moss_sample_counts(h, m, 0, K, seed, counts, stream)
        out = []
        for _ in range(reps):
            l2_flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            moss.moss_sample_counts(h, m, 0, K, seed, counts, stream)
            b.record(stream)
            torch.cuda.synchronize()
            out.append(a.elapsed_time(b))
        times[m] = (K, statistics.median(out))
    return times


NAMES = {0: "MOSS4", 1: "T5", 2: "PATH5", 3: "MOSS4MIN"}


def roofline(workload, rp, probe_name, times, methods, l2_bytes, gather, peaks):
    """The roofline object of the slowest sampling call.  Its achieved rate
    is algorithmic sectors per sample (tests/golden/sectors_<workload>.json)
    x 32 B x samples per call / the call's CUDA-event time.  When the tables
    the call reads fit the L2 the bound is the L2's random-sector rate,
    measured in the same run by moss_gather_rate on a 64 MiB buffer;
    otherwise the HBM copy peak of MEASURED_PEAKS.json, with the HBM
    random-access rate (a 4 GiB buffer) beside it.  The other ceiling is kept
    as a labelled second fraction."""
    spath = os.path.join(ROOT, "tests", "golden", f"sectors_{workload}.json")
    if not os.path.exists(spath):
        return None
    sect = json.load(open(spath))
    dom = max(times, key=lambda m: times[m][1])
    key = f"{NAMES[dom]}_{probe_name}"
    if key not in sect:
        return None
    K, tms = times[dom]
    spb = sect[key]["sectors_per_sample"]
    ach = spb * 32.0 * K / (tms / 1000.0) / 1e9
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    hbm_src = "measured (MEASURED_PEAKS.json copy)" if "hbm_gbs" in peaks else "fallback 6.8 TB/s"
    ws = sampler_tables_bytes(rp, probe_name, methods)
    l2_rate, hbm_rate = gather
    tb, how = small_case_traffic(workload, key, K)
    out = {"kernel": f"k_sample<{dom}> ({NAMES[dom]}, {probe_name} probes)", "achieved": ach, "unit": "GB/s",
           "traffic": tb, "traffic_scaling": how, "algorithmic_bytes_per_sample": spb * 32.0,
           "samples_per_launch": K, "launch_ms": tms, "kernel_times_ms": {NAMES[m]: times[m][1] for m in times},
           "tables_bytes": ws, "l2_bytes": l2_bytes,
           "gather_ceiling": {"unit": "GB/s", "l2_resident_64MiB": l2_rate, "hbm_4GiB": hbm_rate}}
    if ws <= l2_bytes:
        out.update({"bound": "l2", "peak": l2_rate,
                    "peak_source": "measured in this run: random 32 B reads of a 64 MiB buffer (moss_gather_rate)",
                    "frac": ach / l2_rate, "hbm_copy_peak": hbm_peak, "frac_of_hbm_copy_peak": ach / hbm_peak})
    else:
        out.update({"bound": "hbm", "peak": hbm_peak, "peak_source": hbm_src, "frac": ach / hbm_peak})
        if tb is not None:
            # a load that misses L2 fills a whole 128 B line (ncu on the gather
            # kernel: 125 B of DRAM per load from 4 GiB), so DRAM bytes / 128
            # are the call's random HBM accesses
            fetch = tb / 128.0 / (tms / 1000.0)
            out["dram_line_fetches_per_s"] = fetch
            out["frac_of_hbm_gather"] = fetch / (hbm_rate * 1e9 / 32.0)
    return out


def run_gpu(args):
    import torch
    import torch.distributed as tdist

    import synth
    import paper_1509_08089_gb300 as moss
    from paper_1509_08089_gb300.dist import estimate_weak, sub_budgets

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    mix = args.mode == "min"
    if mix:
        args.k = 4
    METRIC, WORKLOAD = describe(args.workload, args.k, mix)
    if world != args.gpus:
        raise SystemExit(f"--gpus {args.gpus} but WORLD_SIZE={world}")
    extras = world == 1 and args.mode == "single" and not args.no_extras
    # the host process pool (CPU baseline, input generation) is spawned before the first GPU call
    pool = None
    cores = os.cpu_count() or 1
    if rank == 0 and world == 1 and (extras or not args.no_cpu_baseline):
        pool = make_pool(cores)
    futures = {}
    if extras:
        futures["config3"] = pool.submit(_workload, "cl_n4m")
        futures["batched"] = [pool.submit(_make_graph, spec) for spec in batch_specs(args.graphs)[0]]
        futures["served"] = [pool.submit(_make_served, spec) for spec in serve_specs(64)]
    torch.cuda.set_device(local)
    dev = local
    if world > 1:
        tdist.init_process_group("nccl", device_id=torch.device(f"cuda:{local}"))
    moss.load()
    k = args.k
    kmask = (1 << k) | (moss.TABLES_4MIN if mix else 0)
    rp, col = synth.workload(args.workload)
    stream = torch.cuda.current_stream(dev)
    rp_d = torch.from_numpy(rp.view(np.int64)).to(f"cuda:{dev}")
    col_d = torch.from_numpy(col.view(np.int32)).to(f"cuda:{dev}")
    rp_h = torch.from_numpy(rp.view(np.int64)).pin_memory()
    col_h = torch.from_numpy(col.view(np.int32)).pin_memory()
    l2_flush = torch.empty(512 << 20, dtype=torch.uint8, device=f"cuda:{dev}")   # > 126 MB L2
    l2_bytes = torch.cuda.get_device_properties(dev).L2_cache_size

    def allreduce(counts: np.ndarray) -> np.ndarray:
        t = torch.from_numpy(counts).to(f"cuda:{dev}")
        tdist.all_reduce(t)
        return t.cpu().numpy()

    probe = {"auto": moss.PROBE_AUTO, "hash": moss.PROBE_HASH, "filter": moss.PROBE_FILTER,
             "search": moss.PROBE_SEARCH}[args.probe]

    rng = RNG_IDS[args.rng]

    methods_main = [m for m, _ in sub_budgets(k, args.budget, mix)]
    order_main = resolved_order(args.vertex_order, rp, resolved_probe(args.probe, rp), methods_main, l2_bytes)

    def step(src_rp, src_col, seed, kk=k, budget=args.budget, order=order_main):
        h = moss.moss_graph_load_csr(src_rp, src_col, device=dev, stream=stream, order=ORDER_IDS[order])
        try:
            moss.moss_set_probe(h, probe)
            moss.moss_set_rng(h, rng)
            if args.vertex_split >= 0:
                moss.moss_set_vertex_split(h, args.vertex_split)
            moss.moss_build_tables(h, (1 << kk) | (moss.TABLES_4MIN if mix else 0), stream)
            if world == 1 and mix:
                K4, Km = (K for _, K in sub_budgets(kk, budget, True))
                r = moss.result_dict(moss.moss_sample_estimate_min(h, K4, Km, seed, stream))
            elif world == 1:
                r = moss.result_dict(moss.moss_sample_estimate(h, kk, budget, seed, stream))
            else:
                class _G:  # the weak-scaling helper wants .handle/.device/.stats()
                    handle, device = h, dev

                    @staticmethod
                    def stats():
                        return moss.moss_graph_stats(h)
                r = estimate_weak(_G, kk, budget, seed, rank, world, allreduce, stream, mix)
        finally:
            moss.moss_graph_free(h)
        return r

    def barrier():
        if world > 1:
            tdist.barrier()

    def timed_steps(src_rp, src_col, nsteps, seed0, **kw):
        """nsteps steps, L2 flushed before each, CUDA events on the stream."""
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(nsteps)]
        barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for i in range(nsteps):
            l2_flush.zero_()                 # evict the previous step's tables from L2
            ev[i][0].record(stream)
            step(src_rp, src_col, seed0 + i, **kw)
            ev[i][1].record(stream)
        torch.cuda.synchronize()
        barrier()
        return [a.elapsed_time(b) for a, b in ev], time.perf_counter() - t0

    for i in range(args.warmup):
        step(rp_d, col_d, args.seed + i)
    torch.cuda.synchronize()
    if futures:
        # inputs of the other terms are generated on the host cores; let that
        # finish before anything is timed
        import concurrent.futures as cf
        cf.wait([futures["config3"], *futures["batched"], *futures["served"]])
    clocks = Clocks(dev)
    clocks.start()
    step_ms, t_wall = timed_steps(rp_d, col_d, args.steps, args.seed + 100)
    clk = clocks.stop()
    ms = sum(step_ms) / len(step_ms)
    if world > 1:
        t = torch.tensor([ms], device=f"cuda:{dev}", dtype=torch.float64)
        tdist.all_reduce(t, op=tdist.ReduceOp.MAX)
        ms = float(t.item())
    samples_per_step = args.budget * world
    value = samples_per_step / (ms / 1000.0)

    # ---- end to end through the public API from pinned host buffers
    e2e_t = []
    for i in range(args.e2e_steps):
        barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        step(rp_h, col_h, args.seed + 200 + i)
        torch.cuda.synchronize()
        barrier()
        e2e_t.append(time.perf_counter() - t0)
    e2e_s = statistics.median(e2e_t)
    if world > 1:
        t = torch.tensor([e2e_s], device=f"cuda:{dev}", dtype=torch.float64)
        tdist.all_reduce(t, op=tdist.ReduceOp.MAX)
        e2e_s = float(t.item())
    h2d = rp.nbytes + col.nbytes
    d2h = __import__("ctypes").sizeof(moss.moss_result)

    # ---- the dominant sampling call alone (the same call as inside the step)
    peaks = peaks_file()
    probe_name = resolved_probe(args.probe, rp)
    h = moss.moss_graph_load_csr(rp_d, col_d, device=dev, stream=stream, order=ORDER_IDS[order_main])
    try:
        moss.moss_set_probe(h, probe)
        moss.moss_set_rng(h, rng)
        if args.vertex_split >= 0:
            moss.moss_set_vertex_split(h, args.vertex_split)
        moss.moss_build_tables(h, kmask, stream)
        times = time_calls(moss, torch, h, k, args.budget, mix, args.seed, stream, l2_flush)
    finally:
        moss.moss_graph_free(h)
    gather = (moss.moss_gather_rate(64 << 20, dev, stream) * 32.0 / 1e9,
              moss.moss_gather_rate(4 << 30, dev, stream) * 32.0 / 1e9)
    roof = roofline(data_key(args.workload, order_main), rp, probe_name, times, methods_main, l2_bytes, gather,
                    peaks)

    out = {
        "metric": METRIC, "value": value, "unit": "samples/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int64", "data": "synthetic",
        "config": bench_config(args, rp, world, WORKLOAD, order_main),
        "e2e": {"value": samples_per_step / e2e_s, "unit": "samples/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "roofline": roof,
        "clocks": clk,
        "gpu_launches": launches_per_step(k, args.budget, mix, probe_name == "filter", *two_levels(args, len(rp) - 1),
                                          ordered=order_main == "degree") * args.steps,
        "wall_s_timed": t_wall,
        "step_ms": step_ms,
    }
    del rp_d, col_d, rp_h, col_h

    if extras:
        # ---- the 34M-edge graph (HBM-resident tables): k = 5, 1e9 samples per step
        rp3, col3 = futures["config3"].result()
        rp3_d = torch.from_numpy(rp3.view(np.int64)).to(f"cuda:{dev}")
        col3_d = torch.from_numpy(col3.view(np.int32)).to(f"cuda:{dev}")
        B3 = 1_000_000_000
        p3 = resolved_probe(args.probe, rp3)
        o3 = resolved_order(args.vertex_order, rp3, p3, [1, 2], l2_bytes)
        for i in range(args.warmup):
            step(rp3_d, col3_d, args.seed + i, budget=B3, order=o3)
        torch.cuda.synchronize()
        c3 = Clocks(dev)
        c3.start()
        ms3, _ = timed_steps(rp3_d, col3_d, args.steps, args.seed + 100, budget=B3, order=o3)
        clk3 = c3.stop()
        h = moss.moss_graph_load_csr(rp3_d, col3_d, device=dev, stream=stream, order=ORDER_IDS[o3])
        try:
            moss.moss_set_probe(h, probe)
            moss.moss_set_rng(h, rng)
            moss.moss_build_tables(h, 1 << 5, stream)
            t3 = time_calls(moss, torch, h, 5, B3, False, args.seed, stream, l2_flush, reps=2)
        finally:
            moss.moss_graph_free(h)
        del rp3_d, col3_d
        m3 = sum(ms3) / len(ms3)
        out["config3"] = {
            "metric": "5-node samples/s at 34M edges", "value": B3 / (m3 / 1000.0), "unit": "samples/s",
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": m3, "step_ms": ms3,
            "config": {"workload": describe("cl_n4m", 5)[1], "budget": B3, "seed": args.seed, "probe": p3,
                       "rng": args.rng, "vertex_order": o3,
                       "l2": "flushed (512 MB write) before every timed step; tables larger than the L2"},
            "roofline": roofline(data_key("cl_n4m", o3), rp3, p3, t3, [1, 2], l2_bytes, gather, peaks),
            "clocks": clk3,
            "gpu_launches": launches_per_step(5, B3, False, p3 == "filter", True, ordered=o3 == "degree") * args.steps}
        out["batched"] = measure_batched(moss, torch, [f.result() for f in futures["batched"]],
                                         batch_specs(args.graphs)[1], args.steps, args.warmup, stream, rng)
        out["served"] = measure_served(moss, [f.result() for f in futures["served"]], args.rate,
                                       args.serve_duration, rng=rng)

    if pool is not None and not args.no_cpu_baseline:
        per_worker, single = calibrate_per_worker(args.workload, k, args.seed, 12.0, mix, rng)
        b, sw, n, wall = oracle_pass(pool, cores, args.workload, k, args.seed, per_worker, mix, rng)
        v, rate = oracle_rate(b, sw, n, args.budget)
        out["cpu_baseline"] = {
            "value": v, "unit": "samples/s", "cores": cores, "kind": "oracle",
            "sample": (f"{n} samples ({'T-5/Path-5 evenly' if k == 5 else ('MOSS-4/MOSS-4Min evenly' if mix else 'MOSS-4')}) over {cores} processes in "
                       f"{sw:.1f} s + table build {b:.2f} s, extrapolated to the {args.budget}-sample budget"),
            "sampling_rate": rate, "single_core_sampling_rate": single}
    if pool is not None:
        pool.shutdown()
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        tdist.destroy_process_group()


# ----------------------------------------------------------------- batch --
def _workload(name):
    sys.path.insert(0, ROOT)
    import synth
    return synth.workload(name)


def _make_graph(spec):
    sys.path.insert(0, ROOT)
    import synth
    kind, n, a, b, seed = spec
    if kind == "cl":
        return synth.chung_lu(n, a, b, min(0.2 * n, 50 * b), seed=seed)
    return synth.rgg(n, a, seed=seed)


def batch_specs(count: int, seed: int = 7):
    """The batched workload: `count` graphs, n log-uniform in [500, 50,000];
    even ones Chung-Lu (exponent 2.0-3.0, mean degree 4-12), odd ones 2-D
    random geometric (mean degree 6-30); k in {4, 5} and a budget
    log-uniform in [1e4, 1e7] per graph.  Returns (graph specs, (k, budget,
    seed) per graph)."""
    rng = np.random.default_rng(seed)
    specs, meta = [], []
    for i in range(count):
        n = int(np.exp(rng.uniform(np.log(500), np.log(50_000))))
        if i % 2 == 0:
            dbar = float(rng.uniform(4.0, 12.0))
            specs.append(("cl", n, float(rng.uniform(2.0, 3.0)), dbar, 10_000 + i))
        else:
            specs.append(("rgg", n, float(rng.uniform(6.0, 30.0)), 0.0, 20_000 + i))
        k = int(rng.choice([4, 5]))
        budget = int(np.exp(rng.uniform(np.log(1e4), np.log(1e7))))
        meta.append((k, budget, int(rng.integers(1, 2**62))))
    return specs, meta


BATCH_WORKLOAD = ("{n} graphs, n 500-50,000 log-uniform, half Chung-Lu exponent 2.0-3.0, half 2-D RGG mean "
                  "degree 6-30, k in {{4,5}}, budgets 1e4-1e7 log-uniform")


def measure_batched(moss, torch, csrs, meta, steps, warmup, stream, rng=0):
    """Every graph's request in one persistent launch (autotuned), timed by
    the host around the synchronous call, against one moss_sample_estimate
    launch per request back to back; counts must agree."""
    t0 = time.perf_counter()
    graphs = [moss.Graph(rp, col, stream=stream, rng=rng) for rp, col in csrs]
    load_s = time.perf_counter() - t0
    total = sum(b for _, b, _ in meta)
    edges = sum(len(col) // 2 for _, col in csrs)
    try:
        with moss.Batch() as batch:
            for g, (k, b, sd) in zip(graphs, meta):
                batch.add(g, k, b, sd)
            tuned = batch.tune(stream)
            for _ in range(warmup):
                batch.run(stream)
            clocks = Clocks(torch.cuda.current_device())
            clocks.start()
            times = []
            for _ in range(steps):
                torch.cuda.synchronize()
                a = time.perf_counter()
                res = batch.run(stream)
                times.append(time.perf_counter() - a)
            clk = clocks.stop()
            tuning = batch.tuning()
        plain = []
        for _ in range(max(1, steps // 4)):
            torch.cuda.synchronize()
            a = time.perf_counter()
            solo = [g.estimate(k, b, sd, stream) for g, (k, b, sd) in zip(graphs, meta)]
            plain.append(time.perf_counter() - a)
        same = all(np.array_equal(r["hits"], q["hits"]) for r, q in zip(res, solo))
    finally:
        for g in graphs:
            g.close()
    tb, tp = statistics.median(times), statistics.median(plain)
    return {"metric": "batched samples/s over many graphs", "value": total / tb, "unit": "samples/s",
            "steps": steps, "warmup": warmup, "ms_per_step": 1000 * tb,
            "timing": "host wall clock around the synchronous batch run (one CUDA graph launch)",
            "config": {"workload": BATCH_WORKLOAD.format(n=len(csrs)), "samples_per_step": total,
                       "edges_total": edges, "tile_samples": tuned, "tuning": tuning,
                       "load_and_build_s": round(load_s, 2)},
            "plain": {"value": total / tp, "ms_per_step": 1000 * tp,
                      "what": "one moss_sample_estimate launch per request, back to back"},
            "speedup_vs_plain": tp / tb, "identical_counts": bool(same), "clocks": clk}


def run_batch(args):
    import torch
    import paper_1509_08089_gb300 as moss

    specs, meta = batch_specs(args.graphs)
    t0 = time.perf_counter()
    with make_pool(os.cpu_count() or 1) as pool:   # spawned before the first GPU call
        csrs = list(pool.map(_make_graph, specs))
    gen_s = time.perf_counter() - t0
    torch.cuda.set_device(0)
    moss.load()
    stream = torch.cuda.current_stream()
    r = measure_batched(moss, torch, csrs, meta, args.steps, args.warmup, stream, RNG_IDS[args.rng])
    r.update({"n_gpus": 1, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
              "data": "synthetic"})
    r["config"]["generation_s"] = round(gen_s, 1)
    print(json.dumps(r), flush=True)


# ----------------------------------------------------------------- serve --
def _make_served(spec):
    sys.path.insert(0, ROOT)
    import synth
    n, gamma, dbar, seed = spec
    return synth.chung_lu(n, gamma, dbar, min(0.1 * n, 30 * dbar), seed=seed)


def serve_specs(count: int, seed: int = 11):
    """`count` Chung-Lu graphs with edge counts log-uniform in [1e4, 1e7]
    (mean degree 8-20, exponent 2.1-2.8)."""
    rng = np.random.default_rng(seed)
    specs = []
    for i in range(count):
        edges = float(np.exp(rng.uniform(np.log(1e4), np.log(1e7))))
        dbar = float(rng.uniform(8.0, 20.0))
        specs.append((max(200, int(2 * edges / dbar)), float(rng.uniform(2.1, 2.8)), dbar, 30_000 + i))
    return specs


def poisson_schedule(rate: float, duration: float, ngraphs: int, eps_lo: float, eps_hi: float, seed: int):
    rng = np.random.default_rng(seed)
    t, out = 0.0, []
    while True:
        t += float(rng.exponential(1.0 / rate))
        if t > duration:
            return out
        out.append((t, int(rng.integers(0, ngraphs)), int(rng.choice([4, 5])), float(rng.uniform(eps_lo, eps_hi)),
                    int(rng.integers(1, 2**62))))


def serve_once(moss, graphs, schedule, config):
    import threading
    with moss.Server(**config) as server:
        gids = [server.add_graph(g) for g in graphs]
        subs = []
        t0 = time.perf_counter()

        def submitter():
            for at, gi, k, eps, sd in schedule:
                delay = t0 + at - time.perf_counter()
                if delay > 0:
                    time.sleep(delay)
                subs.append(server.submit(gids[gi], k, target_rse=eps, seed=sd))

        th = threading.Thread(target=submitter)
        th.start()
        th.join()
        stats = [server.wait(rid, 3600.0)[1] for rid in subs]
        info = server.stats()
    lat = np.array([x["latency_s"] for x in stats]) * 1000.0
    samples = sum(x["budget"] for x in stats)
    return {"p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "mean_ms": float(lat.mean()), "requests": len(stats), "samples": int(samples),
            "samples_per_s": samples / info["span_s"] if info["span_s"] else None,
            "gpu_busy_frac": info["busy_s"] / info["span_s"] if info["span_s"] else None,
            "launches": int(info["ticks"])}


SERVE_COMMON = dict(min_budget=10_000, max_budget=10_000_000, pilot_samples=20_000)
SERVED_CFG = dict(max_active=512, tick_samples=100_000_000, tile_samples=4096, **SERVE_COMMON)
# one request per launch: one slot, a tick as large as the largest budget
PLAIN_CFG = dict(max_active=1, tick_samples=10_000_000, tile_samples=4096, **SERVE_COMMON)


def measure_served(moss, csrs, rate: float, duration: float, eps=(0.01, 0.05), rng=0):
    """A Poisson stream of target-error requests over resident graphs, served
    with continuous batching and, on the same stream, one request per
    launch; each with its own clock record."""
    import torch
    graphs = [moss.Graph(rp, col, rng=rng) for rp, col in csrs]
    edges = sum(len(col) // 2 for _, col in csrs)
    try:
        sched = poisson_schedule(rate, duration, len(graphs), eps[0], eps[1], seed=5)
        serve_once(moss, graphs, sched[: max(1, len(sched) // 20)], SERVED_CFG)   # warm-up
        c = Clocks(torch.cuda.current_device())
        c.start()
        served = serve_once(moss, graphs, sched, SERVED_CFG)
        served["clocks"] = c.stop()
        c = Clocks(torch.cuda.current_device())
        c.start()
        plain = serve_once(moss, graphs, sched, PLAIN_CFG)
        plain["clocks"] = c.stop()
    finally:
        for g in graphs:
            g.close()
    return {"metric": "served p99 ms vs plain", "value": served["p99_ms"], "unit": "ms", "higher_is_better": False,
            "config": {"workload": (f"Poisson {rate:.0f} req/s for {duration} s over {len(graphs)} resident "
                                    f"Chung-Lu graphs ({edges} edges total, 1e4-1e7 each); k in {{4,5}}; target "
                                    f"relative SE {eps[0]:.0%}-{eps[1]:.0%}, budget from the variance formula "
                                    "after a 2e4-sample pilot, clamped to [1e4, 1e7]; admission by free HBM"),
                       "served": SERVED_CFG, "plain": PLAIN_CFG},
            "served": served, "plain": plain,
            "p99_speedup_vs_plain": plain["p99_ms"] / served["p99_ms"] if served["p99_ms"] else None}


def run_serve(args):
    import torch
    import paper_1509_08089_gb300 as moss

    t0 = time.perf_counter()
    with make_pool(os.cpu_count() or 1) as pool:
        csrs = list(pool.map(_make_served, serve_specs(64)))
    gen_s = time.perf_counter() - t0
    torch.cuda.set_device(0)
    moss.load()
    runs = {name: measure_served(moss, csrs, args.rate, args.duration, eps, RNG_IDS[args.rng])
            for name, eps in (("mixed", (0.01, 0.05)), ("rse_1pct", (0.01, 0.01)))}
    r = dict(runs["mixed"])
    r.update({"n_gpus": 1, "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
              "runs": runs})
    r["config"]["generation_s"] = round(gen_s, 1)
    print(json.dumps(r), flush=True)


def run_call(args):
    """Sampling calls (moss_sample_counts) of each method and size on the
    workload's graph, W untimed and K timed each, the L2 flushed before every
    call; one JSON line with the median CUDA-event time of each.  The launch
    order is fixed (methods in turn, sizes in turn, warm-up calls first), so a
    profiler's launch list maps onto the calls."""
    import torch
    import synth
    import paper_1509_08089_gb300 as moss
    rp, col = synth.workload(args.workload)
    torch.cuda.set_device(0)
    moss.load()
    stream = torch.cuda.current_stream()
    methods = [int(x) for x in args.methods.split(",")]
    counts = [int(x) for x in args.counts.split(",")]
    probe = {"auto": moss.PROBE_AUTO, "hash": moss.PROBE_HASH, "filter": moss.PROBE_FILTER,
             "search": moss.PROBE_SEARCH}[args.probe]
    kmask = (1 << 4) | (1 << 5) | (moss.TABLES_4MIN if 3 in methods else 0)
    l2_flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")
    out = {}
    vsplit = args.vertex_split if args.vertex_split >= 0 else None
    order = resolved_order(args.vertex_order, rp, resolved_probe(args.probe, rp), methods,
                           torch.cuda.get_device_properties(0).L2_cache_size)
    with moss.Graph(rp, col, stream=stream, k_mask=kmask, probe=probe, rng=RNG_IDS[args.rng], vsplit=vsplit,
                    order=ORDER_IDS[order]) as g:
        buf = torch.zeros(22, dtype=torch.int64, device="cuda")
        for m in methods:
            for c in counts:
                ms = []
                for i in range(args.warmup + args.steps):
                    l2_flush.zero_()
                    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    a.record(stream)
                    moss.moss_sample_counts(g.handle, m, 0, c, args.seed, buf, stream)
                    b.record(stream)
                    torch.cuda.synchronize()
                    if i >= args.warmup:
                        ms.append(a.elapsed_time(b))
                out[f"{NAMES[m]}@{c}"] = {"ms": statistics.median(ms), "samples_per_s": c / statistics.median(ms) * 1e3}
    print(json.dumps({"metric": "samples/s of one sampling call", "workload": describe(args.workload, 5)[1],
                      "probe": resolved_probe(args.probe, rp), "rng": args.rng, "vertex_order": order,
                      "steps": args.steps,
                      "warmup": args.warmup, "calls": out}), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.mode == "call":
        run_call(args)
    elif args.mode == "batch":
        run_batch(args)
    elif args.mode == "serve":
        run_serve(args)
    else:
        run_gpu(args)   # single and min


if __name__ == "__main__":
    main()
