"""GB300 Moss motif sampler -- Python binding of libmoss.so (include/moss.h).

A thin ctypes layer: every function marshals its arguments and calls the C
ABI of the same name; all computation (validation, weights, alias tables,
sampling, counting, estimators) runs in the library's CUDA kernels.  There is
no CPU fallback: if ``libmoss.so`` is missing or cannot load, every call
raises.  Build it with ``python -m paper_1509_08089_gb300.build``.

Arrays may be numpy arrays (host memory) or torch tensors (host or CUDA).
``stream`` is a ``torch.cuda.Stream``, a raw ``cudaStream_t`` integer, or None
for torch's current stream on the graph's device (legacy default stream when
torch is unavailable).
"""
from __future__ import annotations

import ctypes
import os
from typing import Any

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libmoss.so")

MOSS_OK, MOSS_EINVAL, MOSS_ENOMEM, MOSS_ECUDA, MOSS_EGRAPH, MOSS_EOVERFLOW, MOSS_ESTATE = 0, -1, -2, -3, -4, -5, -6
MOSS_EBUSY = -7
MOSS4, T5, PATH5, MOSS4MIN = 0, 1, 2, 3
PROBE_SEARCH, PROBE_HASH, PROBE_FILTER, PROBE_AUTO = 0, 1, 2, 3
RNG_SPLITMIX64, RNG_PHILOX4X32 = 0, 1
VERTEX_SPLIT_DEFAULT, VERTEX_SPLIT_MID, VERTEX_ONE_LEVEL = 20, 12, 64
NSLOTS = 22
TABLES_4MIN = 1 << 6
TABLE_VERT, TABLE_SLOT, TABLE_ACC, TABLE_SEED0, TABLE_GAMMA0 = 0, 1, 2, 3, 6
TABLE_MIN_SEED, TABLE_MIN_GAMMA, TABLE_MIN_VERT, TABLE_MIN_SLOT, TABLE_MIN_LIST = 9, 10, 11, 12, 13
TABLE_FILTER = 14
TABLE_MIN_PICK = 15
TABLE_HUB_LIST = 16
TABLE_HUB_BITS = 17
TABLE_ORDER = 18
ORDER_INPUT, ORDER_DEGREE = 0, 1


class moss_stats(ctypes.Structure):
    _fields_ = [("n", ctypes.c_uint32), ("nnz", ctypes.c_uint64), ("d_max", ctypes.c_uint32),
                ("gamma", (ctypes.c_uint64 * 2) * 4), ("lambda3", ctypes.c_uint64 * 2),
                ("lambda4", ctypes.c_uint64 * 2), ("gamma_d", ctypes.c_double * 4),
                ("lambda3_d", ctypes.c_double), ("lambda4_d", ctypes.c_double)]


class moss_result(ctypes.Structure):
    _fields_ = [("k", ctypes.c_int), ("n_classes", ctypes.c_int), ("K", ctypes.c_uint64 * 2),
                ("hits", (ctypes.c_uint64 * NSLOTS) * 2), ("est", ctypes.c_double * NSLOTS),
                ("var", ctypes.c_double * NSLOTS), ("lambda_", (ctypes.c_double * NSLOTS) * 2),
                ("triangles", ctypes.c_double), ("triangles_var", ctypes.c_double),
                ("conc", ctypes.c_double * NSLOTS)]


class moss_batch_tuning(ctypes.Structure):
    _fields_ = [("tile_samples", ctypes.c_uint32), ("threads_per_block", ctypes.c_int),
                ("blocks_per_sm", ctypes.c_int), ("tuned", ctypes.c_int), ("graphs", ctypes.c_int),
                ("graphs_search", ctypes.c_int), ("graphs_hash", ctypes.c_int), ("graphs_filter", ctypes.c_int),
                ("run_s", ctypes.c_double)]


class moss_server_config(ctypes.Structure):
    _fields_ = [("max_active", ctypes.c_int), ("tick_samples", ctypes.c_uint64), ("tile_samples", ctypes.c_uint32),
                ("pilot_samples", ctypes.c_uint64), ("min_budget", ctypes.c_uint64), ("max_budget", ctypes.c_uint64),
                ("reserve_bytes", ctypes.c_uint64)]


class moss_request_stats(ctypes.Structure):
    _fields_ = [("budget", ctypes.c_uint64), ("latency_s", ctypes.c_double), ("queue_s", ctypes.c_double),
                ("ticks", ctypes.c_uint64)]


class moss_server_info(ctypes.Structure):
    _fields_ = [("ticks", ctypes.c_uint64), ("samples", ctypes.c_uint64), ("completed", ctypes.c_uint64),
                ("pending", ctypes.c_uint64), ("active", ctypes.c_uint64), ("busy_s", ctypes.c_double),
                ("span_s", ctypes.c_double)]


class MossError(RuntimeError):
    def __init__(self, status: int, detail: str):
        super().__init__(f"{detail} (status {status})")
        self.status = status


_lib = None
_vp = ctypes.c_void_p
_u64 = ctypes.c_uint64


def load():
    """Load libmoss.so (raises if it is absent: no fallback exists)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is not built; run python -m paper_1509_08089_gb300.build")
    lib = ctypes.CDLL(LIB_PATH)
    sig = {
        "moss_graph_load_csr": ([_vp, ctypes.c_int, _vp, ctypes.c_uint32, _u64, ctypes.c_int, _vp,
                                 ctypes.POINTER(_vp)], ctypes.c_int),
        "moss_graph_load_csr_order": ([_vp, ctypes.c_int, _vp, ctypes.c_uint32, _u64, ctypes.c_int, ctypes.c_int,
                                       _vp, ctypes.POINTER(_vp)], ctypes.c_int),
        "moss_build_tables": ([_vp, ctypes.c_uint, _vp], ctypes.c_int),
        "moss_set_probe": ([_vp, ctypes.c_int], ctypes.c_int),
        "moss_set_rng": ([_vp, ctypes.c_int], ctypes.c_int),
        "moss_set_vertex_split": ([_vp, ctypes.c_int], ctypes.c_int),
        "moss_vertex_levels": ([_vp, ctypes.c_int, ctypes.POINTER(ctypes.c_uint32), ctypes.POINTER(ctypes.c_uint64)],
                               ctypes.c_int),
        "moss_get_rng": ([_vp], ctypes.c_int),
        "moss_sample_estimate": ([_vp, ctypes.c_int, _u64, _u64, _vp, ctypes.POINTER(moss_result)], ctypes.c_int),
        "moss_sample_counts": ([_vp, ctypes.c_int, _u64, _u64, _u64, _vp, _vp], ctypes.c_int),
        "moss_sample_records": ([_vp, ctypes.c_int, _u64, _u64, _u64, _vp, _vp, _vp], ctypes.c_int),
        "moss_sample_counts_noalloc": ([_vp, ctypes.c_int, _u64, _u64, _u64, _vp, _vp], ctypes.c_int),
        "moss_finalize": ([_vp, ctypes.c_int, _vp, _vp, _vp, ctypes.POINTER(moss_result)], ctypes.c_int),
        "moss_sample_estimate_min": ([_vp, _u64, _u64, _u64, _vp, ctypes.POINTER(moss_result)], ctypes.c_int),
        "moss_finalize_min": ([_vp, _vp, _vp, _vp, _vp, ctypes.POINTER(moss_result)], ctypes.c_int),
        "moss_graph_stats": ([_vp, ctypes.POINTER(moss_stats)], ctypes.c_int),
        "moss_covariance": ([_vp, ctypes.c_int, _vp, _vp, _vp, _vp, ctypes.POINTER(moss_result)], ctypes.c_int),
        "moss_table_export": ([_vp, ctypes.c_int, _vp, _u64], ctypes.c_int),
        "moss_graph_free": ([_vp], None),
        "moss_strerror": ([ctypes.c_int], ctypes.c_char_p),
        "moss_last_error_detail": ([], ctypes.c_char_p),
        "moss_version": ([], ctypes.c_char_p),
        "moss_class_tables": ([ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p], ctypes.c_int),
        "moss_batch_create": ([ctypes.c_int, ctypes.POINTER(_vp)], ctypes.c_int),
        "moss_batch_add": ([_vp, _vp, ctypes.c_int, _u64, _u64, ctypes.POINTER(ctypes.c_int)], ctypes.c_int),
        "moss_batch_add_min": ([_vp, _vp, _u64, _u64, _u64, ctypes.POINTER(ctypes.c_int)], ctypes.c_int),
        "moss_batch_size": ([_vp], ctypes.c_int),
        "moss_batch_clear": ([_vp], ctypes.c_int),
        "moss_batch_set_tile": ([_vp, ctypes.c_uint32], ctypes.c_int),
        "moss_batch_tile": ([_vp], ctypes.c_uint32),
        "moss_batch_run": ([_vp, _vp, ctypes.POINTER(moss_result)], ctypes.c_int),
        "moss_batch_tune": ([_vp, _vp, ctypes.POINTER(ctypes.c_uint32)], ctypes.c_int),
        "moss_batch_set_launch": ([_vp, ctypes.c_int, ctypes.c_int], ctypes.c_int),
        "moss_batch_set_graph_probe": ([_vp, _vp, ctypes.c_int], ctypes.c_int),
        "moss_batch_get_tuning": ([_vp, ctypes.POINTER(moss_batch_tuning)], ctypes.c_int),
        "moss_batch_free": ([_vp], None),
        "moss_server_default_config": ([ctypes.POINTER(moss_server_config)], None),
        "moss_server_create": ([ctypes.c_int, ctypes.POINTER(moss_server_config), ctypes.POINTER(_vp)], ctypes.c_int),
        "moss_server_add_graph": ([_vp, _vp, ctypes.POINTER(ctypes.c_int)], ctypes.c_int),
        "moss_server_submit": ([_vp, ctypes.c_int, ctypes.c_int, _u64, ctypes.c_double, _u64,
                                ctypes.POINTER(ctypes.c_uint64)], ctypes.c_int),
        "moss_server_submit_min": ([_vp, ctypes.c_int, _u64, _u64, _u64, ctypes.POINTER(ctypes.c_uint64)],
                                   ctypes.c_int),
        "moss_server_wait": ([_vp, _u64, ctypes.c_double, ctypes.POINTER(moss_result),
                              ctypes.POINTER(moss_request_stats)], ctypes.c_int),
        "moss_server_stats": ([_vp, ctypes.POINTER(moss_server_info)], ctypes.c_int),
        "moss_server_free": ([_vp], None),
        "moss_budget_for_target": ([ctypes.c_int, _vp, _vp, ctypes.c_double, _u64, _u64], ctypes.c_uint64),
        "moss_budget_for_target_min": ([_vp, _vp, ctypes.c_double, _u64, _u64], ctypes.c_uint64),
        "moss_server_submit_min_target": ([_vp, ctypes.c_int, ctypes.c_double, _u64,
                                           ctypes.POINTER(ctypes.c_uint64)], ctypes.c_int),
        "moss_gather_rate": ([_u64, ctypes.c_int, _vp, ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    _lib = lib
    return lib


def _check(rc: int):
    if rc != MOSS_OK:
        lib = load()
        raise MossError(rc, f"{lib.moss_strerror(rc).decode()}: {lib.moss_last_error_detail().decode()}")


def _ptr(x: Any) -> int | None:
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be contiguous")
        return x.ctypes.data
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return x.data_ptr()
    if isinstance(x, int):
        return x
    raise TypeError(f"unsupported buffer type {type(x)}")


def _stream(stream, device: int | None = None) -> int | None:
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return torch.cuda.current_stream(device).cuda_stream
        except Exception:
            pass
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


# ------------------------------------------------------------ C ABI calls --
def moss_version() -> str:
    return load().moss_version().decode()


def moss_class_tables():
    """(class4[64], class5[1024], centred[4096]) as uint8 arrays (host only)."""
    c4 = np.zeros(64, dtype=np.uint8)
    c5 = np.zeros(1024, dtype=np.uint8)
    cc = np.zeros(4096, dtype=np.uint8)
    _check(load().moss_class_tables(c4.ctypes.data, c5.ctypes.data, cc.ctypes.data))
    return c4, c5, cc


def moss_gather_rate(nbytes: int, device: int = 0, stream=None) -> float:
    """Random 32-byte sector reads per second sustained over a buffer of
    nbytes (see include/moss.h: the samplers' gather ceiling)."""
    out = ctypes.c_double(0.0)
    _check(load().moss_gather_rate(int(nbytes), int(device), _stream(stream, device), ctypes.byref(out)))
    return out.value


def moss_strerror(status: int) -> str:
    return load().moss_strerror(status).decode()


def moss_last_error_detail() -> str:
    return load().moss_last_error_detail().decode()


def moss_graph_load_csr(row_ptr, col, n: int | None = None, device: int = 0, stream=None,
                        order: int = ORDER_INPUT) -> int:
    """Copy a CSR graph (host or device arrays) to the device; returns the
    handle.  order: ORDER_INPUT keeps the input ids, ORDER_DEGREE renumbers
    the vertices by degree key (moss_graph_load_csr_order)."""
    lib = load()
    is64 = int(getattr(row_ptr, "dtype", None) in (np.uint64, np.int64) or str(getattr(row_ptr, "dtype", "")) in
               ("torch.int64", "torch.uint64"))
    if n is None:
        n = len(row_ptr) - 1
    nnz = len(col)
    out = _vp()
    _check(lib.moss_graph_load_csr_order(_ptr(row_ptr), is64, _ptr(col) if nnz else None, n, nnz, order, device,
                                         _stream(stream, device), ctypes.byref(out)))
    return out.value


def moss_graph_load_csr_order(row_ptr, col, order: int, n: int | None = None, device: int = 0, stream=None) -> int:
    """moss_graph_load_csr with the internal vertex order (ORDER_INPUT, ORDER_DEGREE)."""
    return moss_graph_load_csr(row_ptr, col, n=n, device=device, stream=stream, order=order)


def moss_build_tables(g: int, k_mask: int = (1 << 4) | (1 << 5), stream=None):
    _check(load().moss_build_tables(g, k_mask, _stream(stream)))


def moss_set_probe(g: int, strategy: int):
    _check(load().moss_set_probe(g, strategy))


def moss_set_rng(g: int, rng: int):
    _check(load().moss_set_rng(g, rng))


def moss_get_rng(g: int) -> int:
    return load().moss_get_rng(g)


def moss_set_vertex_split(g: int, split: int):
    _check(load().moss_set_vertex_split(g, split))


def moss_vertex_levels(g: int, which: int) -> tuple[int, int]:
    """(heavy columns, light-level bound) of vertex table which."""
    nh, tl = ctypes.c_uint32(0), ctypes.c_uint64(0)
    _check(load().moss_vertex_levels(g, which, ctypes.byref(nh), ctypes.byref(tl)))
    return nh.value, tl.value


def moss_sample_estimate(g: int, k: int, budget: int, seed: int, stream=None) -> moss_result:
    r = moss_result()
    _check(load().moss_sample_estimate(g, k, budget, seed, _stream(stream), ctypes.byref(r)))
    return r


def moss_sample_counts(g: int, method: int, first: int, count: int, seed: int, counts_dev, stream=None):
    _check(load().moss_sample_counts(g, method, first, count, seed, _stream(stream), _ptr(counts_dev)))


def moss_sample_counts_noalloc(g: int, method: int, first: int, count: int, seed: int, counts_dev, stream=None):
    """moss_sample_counts for callers that may not allocate device memory:
    the per-block partial counts live in a fixed array inside the library."""
    _check(load().moss_sample_counts_noalloc(g, method, first, count, seed, _stream(stream), _ptr(counts_dev)))


def moss_sample_records(g: int, method: int, first: int, count: int, seed: int, classes_dev, verts_dev=None,
                        stream=None):
    _check(load().moss_sample_records(g, method, first, count, seed, _stream(stream), _ptr(classes_dev),
                                      _ptr(verts_dev)))


def moss_finalize(g: int, k: int, K, hits, stream=None) -> moss_result:
    Ka = np.ascontiguousarray(K, dtype=np.uint64)
    Ha = np.ascontiguousarray(hits, dtype=np.uint64).reshape(2 * NSLOTS)
    r = moss_result()
    _check(load().moss_finalize(g, k, _ptr(Ka), _ptr(Ha), _stream(stream), ctypes.byref(r)))
    return r


def moss_sample_estimate_min(g: int, budget: int, budget_min: int, seed: int, stream=None) -> moss_result:
    """MOSS-4 (K = budget) mixed with MOSS-4Min (K-check = budget_min)."""
    r = moss_result()
    _check(load().moss_sample_estimate_min(g, budget, budget_min, seed, _stream(stream), ctypes.byref(r)))
    return r


def moss_finalize_min(g: int, K, hits, stream=None, covariance: bool = False):
    """The MOSS-4 + MOSS-4Min mix from counts; with covariance=True returns
    (22 x 22 covariance matrix, result)."""
    Ka = np.ascontiguousarray(K, dtype=np.uint64)
    Ha = np.ascontiguousarray(hits, dtype=np.uint64).reshape(2 * NSLOTS)
    cov = np.zeros((NSLOTS, NSLOTS), dtype=np.float64) if covariance else None
    r = moss_result()
    _check(load().moss_finalize_min(g, _ptr(Ka), _ptr(Ha), _stream(stream), _ptr(cov), ctypes.byref(r)))
    return (cov, r) if covariance else r


def moss_covariance(g: int, k: int, K, hits, stream=None):
    """(22 x 22 covariance matrix, result) of the estimates of these counts."""
    Ka = np.ascontiguousarray(K, dtype=np.uint64)
    Ha = np.ascontiguousarray(hits, dtype=np.uint64).reshape(2 * NSLOTS)
    cov = np.zeros((NSLOTS, NSLOTS), dtype=np.float64)
    r = moss_result()
    _check(load().moss_covariance(g, k, _ptr(Ka), _ptr(Ha), _stream(stream), _ptr(cov), ctypes.byref(r)))
    return cov, result_dict(r)


def moss_graph_stats(g: int) -> moss_stats:
    s = moss_stats()
    _check(load().moss_graph_stats(g, ctypes.byref(s)))
    return s


def moss_table_export(g: int, table: int, out: np.ndarray):
    _check(load().moss_table_export(g, table, _ptr(out), out.nbytes))
    return out


def moss_graph_free(g: int):
    if g:
        load().moss_graph_free(g)


def moss_batch_create(device: int = 0) -> int:
    out = _vp()
    _check(load().moss_batch_create(device, ctypes.byref(out)))
    return out.value


def moss_batch_add(b: int, g: int, k: int, budget: int, seed: int) -> int:
    idx = ctypes.c_int(-1)
    _check(load().moss_batch_add(b, g, k, budget, seed, ctypes.byref(idx)))
    return idx.value


def moss_batch_add_min(b: int, g: int, budget: int, budget_min: int, seed: int) -> int:
    idx = ctypes.c_int(-1)
    _check(load().moss_batch_add_min(b, g, budget, budget_min, seed, ctypes.byref(idx)))
    return idx.value


def moss_batch_size(b: int) -> int:
    return load().moss_batch_size(b)


def moss_batch_clear(b: int):
    _check(load().moss_batch_clear(b))


def moss_batch_set_tile(b: int, tile_samples: int):
    _check(load().moss_batch_set_tile(b, tile_samples))


def moss_batch_tile(b: int) -> int:
    return load().moss_batch_tile(b)


def moss_batch_run(b: int, stream=None) -> list:
    n = load().moss_batch_size(b)
    arr = (moss_result * max(n, 1))()
    _check(load().moss_batch_run(b, _stream(stream), arr))
    return [arr[i] for i in range(n)]


def moss_batch_tune(b: int, stream=None) -> int:
    c = ctypes.c_uint32(0)
    _check(load().moss_batch_tune(b, _stream(stream), ctypes.byref(c)))
    return c.value


def moss_batch_set_launch(b: int, threads_per_block: int, blocks_per_sm: int = 0):
    _check(load().moss_batch_set_launch(b, threads_per_block, blocks_per_sm))


def moss_batch_set_graph_probe(b: int, g: int, strategy: int):
    _check(load().moss_batch_set_graph_probe(b, g, strategy))


def moss_batch_get_tuning(b: int) -> moss_batch_tuning:
    t = moss_batch_tuning()
    _check(load().moss_batch_get_tuning(b, ctypes.byref(t)))
    return t


def moss_batch_free(b: int):
    if b:
        load().moss_batch_free(b)


def moss_server_default_config() -> moss_server_config:
    c = moss_server_config()
    load().moss_server_default_config(ctypes.byref(c))
    return c


def moss_server_create(device: int = 0, config: moss_server_config | None = None) -> int:
    out = _vp()
    _check(load().moss_server_create(device, ctypes.byref(config) if config is not None else None, ctypes.byref(out)))
    return out.value


def moss_server_add_graph(s: int, g: int) -> int:
    gid = ctypes.c_int(-1)
    _check(load().moss_server_add_graph(s, g, ctypes.byref(gid)))
    return gid.value


def moss_server_submit(s: int, graph_id: int, k: int, budget: int = 0, target_rse: float = 0.0, seed: int = 1) -> int:
    rid = ctypes.c_uint64(0)
    _check(load().moss_server_submit(s, graph_id, k, budget, target_rse, seed, ctypes.byref(rid)))
    return rid.value


def moss_server_submit_min(s: int, graph_id: int, budget: int, budget_min: int, seed: int = 1) -> int:
    rid = ctypes.c_uint64(0)
    _check(load().moss_server_submit_min(s, graph_id, budget, budget_min, seed, ctypes.byref(rid)))
    return rid.value


def moss_server_wait(s: int, request_id: int, timeout_s: float = 600.0):
    r = moss_result()
    st = moss_request_stats()
    _check(load().moss_server_wait(s, request_id, timeout_s, ctypes.byref(r), ctypes.byref(st)))
    return r, st


def moss_server_stats(s: int) -> moss_server_info:
    i = moss_server_info()
    _check(load().moss_server_stats(s, ctypes.byref(i)))
    return i


def moss_server_free(s: int):
    if s:
        load().moss_server_free(s)


def moss_budget_for_target(k: int, K, hits, target: float, min_budget: int, max_budget: int) -> int:
    Ka = np.ascontiguousarray(K, dtype=np.uint64)
    Ha = np.ascontiguousarray(hits, dtype=np.uint64).reshape(2 * NSLOTS)
    return int(load().moss_budget_for_target(k, _ptr(Ka), _ptr(Ha), target, min_budget, max_budget))


def moss_budget_for_target_min(K, hits, target: float, min_budget: int, max_budget: int) -> int:
    Ka = np.ascontiguousarray(K, dtype=np.uint64)
    Ha = np.ascontiguousarray(hits, dtype=np.uint64)
    return int(load().moss_budget_for_target_min(_ptr(Ka), _ptr(Ha), target, min_budget, max_budget))


def moss_server_submit_min_target(s: int, graph_id: int, target_rse: float, seed: int = 1) -> int:
    rid = ctypes.c_uint64(0)
    _check(load().moss_server_submit_min_target(s, graph_id, target_rse, seed, ctypes.byref(rid)))
    return rid.value


class Server:
    """Owning wrapper of a request server (see moss_server_* in include/moss.h)."""

    def __init__(self, device: int = 0, **config):
        cfg = moss_server_default_config()
        for key, val in config.items():
            setattr(cfg, key, val)
        self.handle = moss_server_create(device, cfg)

    def add_graph(self, graph: "Graph") -> int:
        return moss_server_add_graph(self.handle, graph.handle)

    def submit(self, graph_id: int, k: int, budget: int = 0, target_rse: float = 0.0, seed: int = 1) -> int:
        return moss_server_submit(self.handle, graph_id, k, budget, target_rse, seed)

    def submit_min(self, graph_id: int, budget: int = 0, budget_min: int = 0, seed: int = 1,
                   target_rse: float = 0.0) -> int:
        """A MOSS-4 + MOSS-4Min request: explicit budgets, or a target
        relative standard error whose pilot sets them."""
        if target_rse > 0.0:
            return moss_server_submit_min_target(self.handle, graph_id, target_rse, seed)
        return moss_server_submit_min(self.handle, graph_id, budget, budget_min, seed)

    def wait(self, request_id: int, timeout_s: float = 600.0):
        r, st = moss_server_wait(self.handle, request_id, timeout_s)
        return result_dict(r), {"budget": st.budget, "latency_s": st.latency_s, "queue_s": st.queue_s,
                                "ticks": st.ticks}

    def stats(self) -> dict:
        i = moss_server_stats(self.handle)
        return {f: getattr(i, f) for f, _ in moss_server_info._fields_}

    def close(self):
        if getattr(self, "handle", None):
            moss_server_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


# ------------------------------------------------------------ convenience --
def result_dict(r: moss_result) -> dict:
    """moss_result as plain Python/numpy values."""
    view = np.ctypeslib.as_array
    return {"k": r.k, "K": (int(r.K[0]), int(r.K[1])),
            "hits": view(r.hits).astype(np.uint64, copy=True),
            "est": view(r.est).copy(), "var": view(r.var).copy(),
            "lam": view(r.lambda_).copy(),
            "triangles": r.triangles, "triangles_var": r.triangles_var, "conc": view(r.conc).copy()}


class Batch:
    """Owning wrapper of a request batch (see moss_batch_* in include/moss.h)."""

    def __init__(self, device: int = 0):
        self.handle = moss_batch_create(device)

    def add(self, graph: "Graph", k: int, budget: int, seed: int) -> int:
        return moss_batch_add(self.handle, graph.handle, k, budget, seed)

    def add_min(self, graph: "Graph", budget: int, budget_min: int, seed: int) -> int:
        return moss_batch_add_min(self.handle, graph.handle, budget, budget_min, seed)

    def run(self, stream=None) -> list[dict]:
        return [result_dict(r) for r in moss_batch_run(self.handle, stream)]

    def tune(self, stream=None) -> int:
        return moss_batch_tune(self.handle, stream)

    def tuning(self) -> dict:
        t = moss_batch_get_tuning(self.handle)
        return {f: getattr(t, f) for f, _ in moss_batch_tuning._fields_}

    def set_launch(self, threads_per_block: int, blocks_per_sm: int = 0):
        moss_batch_set_launch(self.handle, threads_per_block, blocks_per_sm)

    def set_probe(self, graph: "Graph", strategy: int):
        moss_batch_set_graph_probe(self.handle, graph.handle, strategy)

    def set_tile(self, tile_samples: int):
        moss_batch_set_tile(self.handle, tile_samples)

    def clear(self):
        moss_batch_clear(self.handle)

    def __len__(self):
        return moss_batch_size(self.handle)

    def close(self):
        if getattr(self, "handle", None):
            moss_batch_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class Graph:
    """Owning wrapper: load, build, sample, free."""

    def __init__(self, row_ptr, col, device: int = 0, stream=None, k_mask: int = (1 << 4) | (1 << 5),
                 probe: int = PROBE_AUTO, rng: int = RNG_SPLITMIX64, vsplit: int | None = None,
                 order: int = ORDER_INPUT):
        """vsplit: heavy level of the vertex tables (0..63, VERTEX_ONE_LEVEL;
        None: the library's default for the graph's size).  order:
        ORDER_INPUT or ORDER_DEGREE (the vertices renumbered by degree key)."""
        self.handle = moss_graph_load_csr(row_ptr, col, device=device, stream=stream, order=order)
        self.device = device
        moss_set_probe(self.handle, probe)
        moss_set_rng(self.handle, rng)
        if vsplit is not None:
            moss_set_vertex_split(self.handle, vsplit)
        self.k_mask = k_mask
        if k_mask:
            moss_build_tables(self.handle, k_mask, stream)

    def set_probe(self, probe: int, stream=None):
        """Switch the probe strategy, building what it needs."""
        moss_set_probe(self.handle, probe)
        if self.k_mask:
            moss_build_tables(self.handle, self.k_mask, stream)

    def set_rng(self, rng: int):
        """Word generator of later samples (RNG_SPLITMIX64 or RNG_PHILOX4X32)."""
        moss_set_rng(self.handle, rng)

    def estimate(self, k: int, budget: int, seed: int, stream=None) -> dict:
        return result_dict(moss_sample_estimate(self.handle, k, budget, seed, stream))

    def estimate_min(self, budget: int, budget_min: int, seed: int, stream=None) -> dict:
        """MOSS-4 with MOSS-4Min (needs k_mask with (1 << 4) | TABLES_4MIN)."""
        return result_dict(moss_sample_estimate_min(self.handle, budget, budget_min, seed, stream))

    def stats(self) -> moss_stats:
        return moss_graph_stats(self.handle)

    def close(self):
        if getattr(self, "handle", None):
            moss_graph_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
