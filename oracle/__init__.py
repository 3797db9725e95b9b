"""CPU oracle of the Moss sampling path -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product library never imports it
and shares no code with it.

Contents
* ``moss_oracle.c`` (compiled with gcc on first use): exact integer vertex
  weights and totals (Table 1), alias tables for WeightRandomVertex
  (Sec. 4.1.3), the counter-form SplitMix64 and Philox4x32-10 word
  schedules, the per-sample steps of
  Algorithm 1 (MOSS-4), Algorithm 2 (MOSS-4Min, Sec. 4.2: the total order,
  N_{u,v}, the weights Gamma-check_v and sigma-check, and c(s), the number
  of 3-paths of a CIS that the method can draw), Algorithm 3 (T-5) and
  Algorithm 4 (Path-5), the motif classifier (Sec. 4.1.2, Table 2) and ESU
  exact enumeration.
* :mod:`oracle.finalize` (numpy, FP64): the estimators and variances of
  Theorems 3, 5, 7, 9 and 10 and the mix estimator (Theorem 1) of MOSS-4
  with MOSS-4Min and of T-5 with Path-5 (Sec. 5.1.3).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

from .finalize import finalize_moss4, finalize_moss4min, finalize_moss5, min_slot, PHI4, PHI5  # noqa: F401

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "moss_oracle.c")
_LIB = os.path.join(_HERE, "libmoss_oracle.so")
_lib = None

MOSS4, T5, PATH5, MOSS4MIN = 0, 1, 2, 3
SPLITMIX64, PHILOX4X32 = 0, 1     # word generators

_u64p = ctypes.POINTER(ctypes.c_uint64)
_u32p = ctypes.POINTER(ctypes.c_uint32)
_u8p = ctypes.POINTER(ctypes.c_uint8)


def build(force: bool = False) -> str:
    """Compile the oracle library with gcc (portable flags)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-ffp-contract=off", "-fPIC", "-shared",
                               "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        lib.oracle_new.argtypes = [ctypes.c_uint32, _u64p, _u32p]
        lib.oracle_new.restype = ctypes.c_void_p
        lib.oracle_new_split.argtypes = [ctypes.c_uint32, _u64p, _u32p, ctypes.c_int]
        lib.oracle_new_split.restype = ctypes.c_void_p
        lib.oracle_set_min_split.argtypes = [ctypes.c_void_p, ctypes.c_int]
        lib.oracle_free.argtypes = [ctypes.c_void_p]
        lib.oracle_totals.argtypes = [ctypes.c_void_p, _u64p]
        lib.oracle_vertex.argtypes = [ctypes.c_void_p, _u64p, _u64p, _u64p, _u64p]
        lib.oracle_vertex_table.argtypes = [ctypes.c_void_p, ctypes.c_int, _u32p, _u64p, _u32p, _u64p, _u64p, _u32p]
        lib.oracle_sigma_table.argtypes = [ctypes.c_void_p, _u64p, _u32p, _u64p]
        lib.oracle_alias_build.argtypes = [ctypes.c_uint64, _u64p, _u64p, _u32p]
        lib.oracle_alias_build.restype = ctypes.c_int
        lib.oracle_splitmix.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
        lib.oracle_splitmix.restype = ctypes.c_uint64
        lib.oracle_classify.argtypes = [ctypes.c_int, ctypes.c_uint32]
        lib.oracle_classify.restype = ctypes.c_int
        lib.oracle_sample_words.argtypes = [ctypes.c_void_p, ctypes.c_int, _u64p, _u32p, ctypes.POINTER(ctypes.c_int)]
        lib.oracle_sample_words.restype = ctypes.c_int
        lib.oracle_run.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64,
                                   _u64p, _u8p, _u32p]
        lib.oracle_run.restype = ctypes.c_int
        lib.oracle_run_rng.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_uint64, ctypes.c_uint64,
                                       ctypes.c_uint64, _u64p, _u8p, _u32p]
        lib.oracle_run_rng.restype = ctypes.c_int
        lib.oracle_philox4x32.argtypes = [_u32p, _u32p, _u32p]
        lib.oracle_words.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_uint64, ctypes.c_uint64, _u64p]
        lib.oracle_esu.argtypes = [ctypes.c_void_p, ctypes.c_int, _u64p]
        lib.oracle_esu.restype = ctypes.c_int
        lib.oracle_build_min.argtypes = [ctypes.c_void_p]
        lib.oracle_build_min.restype = ctypes.c_int
        lib.oracle_min_total.argtypes = [ctypes.c_void_p, _u64p]
        lib.oracle_min_tables.argtypes = [ctypes.c_void_p, _u32p, _u64p, _u64p, _u32p, _u64p]
        _lib = lib
    return _lib


def _p(a: np.ndarray, t):
    return a.ctypes.data_as(t)


def _u128(lohi) -> int:
    return int(lohi[0]) | (int(lohi[1]) << 64)


def splitmix64(seed: int, k: int) -> int:
    """Output number k >= 1 of SplitMix64 seeded with seed."""
    return int(_load().oracle_splitmix(seed % (1 << 64), k % (1 << 64)))


def sample_words(method: int, seed: int, s: int, n: int = 16, rng: int = SPLITMIX64) -> list[int]:
    """Words x_0 .. x_{n-1} of sample s of a method: SplitMix64 output
    (4 s + method) 16 + i + 1 under seed; or, with rng=PHILOX4X32, words 2b,
    2b+1 from Philox4x32-10 block (s lo, s hi, method, b) under the key
    (seed lo, seed hi)."""
    if rng == SPLITMIX64:
        return [splitmix64(seed, (4 * s + method) * 16 + i + 1) for i in range(n)]
    x = np.zeros(16, dtype=np.uint64)
    _load().oracle_words(rng, method, seed % (1 << 64), s % (1 << 64), _p(x, _u64p))
    return [int(v) for v in x[:n]]


def philox4x32(counter, key) -> list[int]:
    """The four 32-bit outputs of Philox4x32-10 for a 4-word counter and a
    2-word key."""
    c = np.array([int(v) for v in counter], dtype=np.uint32)
    k = np.array([int(v) for v in key], dtype=np.uint32)
    o = np.zeros(4, dtype=np.uint32)
    _load().oracle_philox4x32(_p(c, _u32p), _p(k, _u32p), _p(o, _u32p))
    return [int(v) for v in o]


def classify(k: int, mask: int) -> int:
    """Motif class (1-based) of the k-vertex graph given by a pair bitmask;
    0 when disconnected."""
    return _load().oracle_classify(k, mask)


def alias_build(weights) -> tuple[list[int], list[int]]:
    """Alias table (thresholds, aliases) of integer weights, by the sweep."""
    m = len(weights)
    w = np.zeros(2 * max(m, 1), dtype=np.uint64)
    for j, x in enumerate(weights):
        x = int(x)
        w[2 * j] = x & ((1 << 64) - 1)
        w[2 * j + 1] = x >> 64
    thr = np.zeros(2 * max(m, 1), dtype=np.uint64)
    alias = np.zeros(max(m, 1), dtype=np.uint32)
    rc = _load().oracle_alias_build(m, _p(w, _u64p), _p(thr, _u64p), _p(alias, _u32p))
    if rc:
        raise MemoryError("oracle_alias_build")
    return [_u128(thr[2 * j:2 * j + 2]) for j in range(m)], [int(a) for a in alias[:m]]


VSPLIT = 20           # heavy vertices of a two-level vertex table: w_v 2^VSPLIT >= W
VSPLIT_MID = 12       # the same from 2^14 vertices on
ONE_LEVEL = 64        # the split value of a single-level vertex table


def default_split(n: int) -> int:
    """Two levels with split 20 from 2^20 vertices on, with split 12 from
    2^14 on, one level below."""
    return VSPLIT if n >= 1 << 20 else (VSPLIT_MID if n >= 1 << 14 else ONE_LEVEL)


def default_split_min(n: int) -> int:
    """The MOSS-4Min table: two levels with split 20 from 2^20 vertices on,
    one level below."""
    return VSPLIT if n >= 1 << 20 else ONE_LEVEL


class OracleGraph:
    """The oracle's view of one graph: weights, tables and the samplers.
    vsplit sets the heavy level of the vertex tables (w_v 2^vsplit >= W;
    ONE_LEVEL: a single table; None: default_split(n), and
    default_split_min(n) for the MOSS-4Min table); vsplit_min overrides the
    MOSS-4Min table's (default: vsplit when that is given)."""

    def __init__(self, row_ptr: np.ndarray, col: np.ndarray, vsplit: int | None = None,
                 vsplit_min: int | None = None):
        self.row_ptr = np.ascontiguousarray(row_ptr, dtype=np.uint64)
        self.col = np.ascontiguousarray(col, dtype=np.uint32)
        self.n = len(self.row_ptr) - 1
        self.nnz = int(self.row_ptr[-1])
        if vsplit_min is None:
            vsplit_min = default_split_min(self.n) if vsplit is None else vsplit
        self.vsplit = vsplit = default_split(self.n) if vsplit is None else vsplit
        self.vsplit_min = vsplit_min
        col_buf = self.col if self.nnz else np.zeros(1, dtype=np.uint32)
        self._ctx = _load().oracle_new_split(self.n, _p(self.row_ptr, _u64p), _p(col_buf, _u32p), vsplit)
        if not self._ctx:
            raise MemoryError("oracle_new")
        if _load().oracle_set_min_split(self._ctx, vsplit_min):
            raise ValueError("vsplit_min out of range")
        t = np.zeros(10, dtype=np.uint64)
        _load().oracle_totals(self._ctx, _p(t, _u64p))
        self.Gamma = [_u128(t[0:2]), _u128(t[2:4]), _u128(t[4:6])]
        self.Lambda3 = _u128(t[6:8])
        self.Lambda4 = _u128(t[8:10])

    def __del__(self):
        ctx = getattr(self, "_ctx", None)
        if ctx:
            _load().oracle_free(ctx)
            self._ctx = None

    # -- tables -------------------------------------------------------------
    def vertex(self):
        n = max(self.n, 1)
        deg = np.zeros(n, dtype=np.uint64)
        S = np.zeros(n, dtype=np.uint64)
        Q = np.zeros(n, dtype=np.uint64)
        g = np.zeros(3 * 2 * n, dtype=np.uint64)
        _load().oracle_vertex(self._ctx, _p(deg, _u64p), _p(S, _u64p), _p(Q, _u64p), _p(g, _u64p))
        gam = [[_u128(g[(l * 2 * n) + 2 * v:(l * 2 * n) + 2 * v + 2]) for v in range(self.n)] for l in range(3)]
        return deg[:self.n], S[:self.n], Q[:self.n], gam

    def vertex_table(self, which: int) -> dict:
        """Two-level vertex table of weight which (0 Gamma, 1 Gamma^(1),
        2 Gamma^(2), 3 Gamma-check), in column order: nh heavy columns, then
        the light ones; per column its vertex (self), threshold (thr, exact),
        quantized threshold T and alias; TL = the light level's word bound."""
        if which == 3:
            self.build_min()
        n = max(self.n, 1)
        nh = np.zeros(1, dtype=np.uint32)
        TL = np.zeros(1, dtype=np.uint64)
        self_ = np.zeros(n, dtype=np.uint32)
        thr = np.zeros(2 * n, dtype=np.uint64)
        T = np.zeros(n, dtype=np.uint64)
        alias = np.zeros(n, dtype=np.uint32)
        _load().oracle_vertex_table(self._ctx, which, _p(nh, _u32p), _p(TL, _u64p), _p(self_, _u32p),
                                    _p(thr, _u64p), _p(T, _u64p), _p(alias, _u32p))
        return {"nh": int(nh[0]), "TL": int(TL[0]), "self": self_[:self.n], "T": T[:self.n],
                "alias": alias[:self.n], "thr": [_u128(thr[2 * v:2 * v + 2]) for v in range(self.n)]}

    def sigma_table(self):
        m = max(self.nnz, 1)
        thr = np.zeros(m, dtype=np.uint64)
        alias = np.zeros(m, dtype=np.uint32)
        acc = np.zeros(m, dtype=np.uint64)
        _load().oracle_sigma_table(self._ctx, _p(thr, _u64p), _p(alias, _u32p), _p(acc, _u64p))
        return thr[:self.nnz], alias[:self.nnz], acc[:self.nnz]

    def build_min(self) -> int:
        """Build the MOSS-4Min tables (Sec. 4.2); returns Gamma-check."""
        if _load().oracle_build_min(self._ctx):
            raise MemoryError("oracle_build_min")
        t = np.zeros(2, dtype=np.uint64)
        _load().oracle_min_total(self._ctx, _p(t, _u64p))
        self.Gamma_min = _u128(t)
        return self.Gamma_min

    def min_tables(self):
        """(ordered lists, d_{v,u} per slot, sigma-check thresholds and
        aliases per slot, Gamma-check_v); the vertex table is vertex_table(3)."""
        self.build_min()
        m, n = max(self.nnz, 1), max(self.n, 1)
        rl = np.zeros(m, dtype=np.uint32)
        rk = np.zeros(m, dtype=np.uint64)
        ct = np.zeros(m, dtype=np.uint64)
        ca = np.zeros(m, dtype=np.uint32)
        g = np.zeros(2 * n, dtype=np.uint64)
        _load().oracle_min_tables(self._ctx, _p(rl, _u32p), _p(rk, _u64p), _p(ct, _u64p), _p(ca, _u32p),
                                  _p(g, _u64p))
        gam = [_u128(g[2 * v:2 * v + 2]) for v in range(self.n)]
        return (rl[:self.nnz], rk[:self.nnz], ct[:self.nnz], ca[:self.nnz], gam)

    # -- sampling -----------------------------------------------------------
    def sample_words(self, method: int, words) -> tuple[list[int], int]:
        if method == MOSS4MIN:
            self.build_min()
        x = np.zeros(16, dtype=np.uint64)
        for i, w in enumerate(words):
            x[i] = int(w)
        verts = np.zeros(5, dtype=np.uint32)
        cls = ctypes.c_int(0)
        rc = _load().oracle_sample_words(self._ctx, method, _p(x, _u64p), _p(verts, _u32p), ctypes.byref(cls))
        if rc:
            raise ValueError("method has zero total weight on this graph")
        return [int(v) for v in verts], cls.value

    def run(self, method: int, seed: int, count: int, first: int = 0, record: bool = False, rng: int = SPLITMIX64):
        """Counts (uint64[22]; [0] = collisions) of samples first..first+count-1.
        With record=True also per-sample classes (uint8) and vertices (uint32[.,5]).
        MOSS-4Min (method 3) counts by (class, c) slot (:func:`min_slot`) and
        records c(s) as the fifth vertex entry.  rng picks the word generator."""
        if method == MOSS4MIN:
            self.build_min()
        counts = np.zeros(22, dtype=np.uint64)
        classes = np.zeros(max(count, 1), dtype=np.uint8) if record else None
        verts = np.zeros((max(count, 1), 5), dtype=np.uint32) if record else None
        rc = _load().oracle_run_rng(self._ctx, method, rng, seed, first, count, _p(counts, _u64p),
                                    _p(classes, _u8p) if record else None,
                                    _p(verts, _u32p) if record else None)
        if rc == -1:
            raise ValueError("method has zero total weight on this graph")
        if rc:
            raise RuntimeError(f"oracle_run failed ({rc})")
        if record:
            return counts, classes[:count], verts[:count]
        return counts

    def esu(self, k: int) -> np.ndarray:
        """Exact counts of connected induced k-subgraphs per class (index 1..)."""
        counts = np.zeros(22, dtype=np.uint64)
        if _load().oracle_esu(self._ctx, k, _p(counts, _u64p)):
            raise ValueError("k must be 4 or 5")
        return counts

    # -- the whole path -----------------------------------------------------
    def estimate(self, k: int, budget: int, seed: int, rng: int = SPLITMIX64, **kw):
        """Sample-and-estimate as the library defines it: k=4 runs MOSS-4 with
        K=budget; k=5 runs T-5 with K1=floor(budget/2) and Path-5 with
        K2=budget-K1 (K1=K2, Sec. 5.1.5)."""
        if k == 4:
            K = budget if self.Gamma[0] > 0 else 0
            m = self.run(MOSS4, seed, K, rng=rng) if K else np.zeros(22, dtype=np.uint64)
            return finalize_moss4(m, K, self.Gamma[0], self.Lambda3, **kw)
        K1 = budget // 2
        K2 = budget - K1
        K1 = K1 if self.Gamma[1] > 0 else 0
        K2 = K2 if self.Gamma[2] > 0 else 0
        m1 = self.run(T5, seed, K1, rng=rng) if K1 else np.zeros(22, dtype=np.uint64)
        m2 = self.run(PATH5, seed, K2, rng=rng) if K2 else np.zeros(22, dtype=np.uint64)
        return finalize_moss5(m1, m2, K1, K2, self.Gamma[1], self.Gamma[2], self.Lambda4, **kw)

    def estimate_min(self, budget: int, budget_min: int, seed: int, rng: int = SPLITMIX64, **kw):
        """MOSS-4 with K = budget and MOSS-4Min with K-check = budget_min on
        the same seed, mixed by Theorem 1 (Sec. 4.2)."""
        Gm = self.build_min()
        K = budget if self.Gamma[0] > 0 else 0
        Km = budget_min if Gm > 0 else 0
        m = self.run(MOSS4, seed, K, rng=rng) if K else np.zeros(22, dtype=np.uint64)
        mm = self.run(MOSS4MIN, seed, Km, rng=rng) if Km else np.zeros(22, dtype=np.uint64)
        return finalize_moss4min(m, mm, K, Km, self.Gamma[0], Gm, self.Lambda3, **kw)
