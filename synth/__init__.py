"""Seeded synthetic graph inputs shared by the oracle, the tests and the bench.

This module holds no part of the sampling method.  It produces simple
undirected graphs as sorted CSR arrays ``(row_ptr: uint64[n+1], col: uint32[nnz])``:

* :func:`chung_lu` -- expected-degree power-law graphs (Miller-Hagberg
  generator), the stand-in for the paper's SNAP graphs (Table 3).
* :func:`rgg` -- 2-D random geometric graphs on the unit torus.
* :func:`from_edges` and the small named families (cycle, complete, star)
  used for the closed-form special cases.

The C generator (``synth.c``) is compiled on first use with gcc into this
directory; :func:`build` does it eagerly.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "synth.c")
_LIB = os.path.join(_HERE, "libsynth.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile ``libsynth.so`` (portable flags, no FMA contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared",
                               "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        lib.synth_generate.argtypes = [ctypes.c_int, ctypes.c_uint32, ctypes.c_double, ctypes.c_double,
                                       ctypes.c_double, ctypes.c_uint64, ctypes.c_int,
                                       ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_void_p)]
        lib.synth_generate.restype = ctypes.c_int
        lib.synth_free.argtypes = [ctypes.c_void_p]
        lib.synth_log.argtypes = [ctypes.c_double]
        lib.synth_log.restype = ctypes.c_double
        lib.synth_exp.argtypes = [ctypes.c_double]
        lib.synth_exp.restype = ctypes.c_double
        _lib = lib
    return _lib


def _generate(kind: int, n: int, gamma: float, dbar: float, dmax: float, seed: int, relabel: bool):
    lib = _load()
    rp = ctypes.c_void_p()
    cl = ctypes.c_void_p()
    rc = lib.synth_generate(kind, n, gamma, dbar, dmax, seed, int(relabel), ctypes.byref(rp), ctypes.byref(cl))
    if rc != 0:
        raise ValueError(f"synth_generate failed (kind={kind}, n={n})")
    try:
        row_ptr = np.ctypeslib.as_array(ctypes.cast(rp, ctypes.POINTER(ctypes.c_uint64)), shape=(n + 1,)).copy()
        nnz = int(row_ptr[-1])
        if nnz:
            col = np.ctypeslib.as_array(ctypes.cast(cl, ctypes.POINTER(ctypes.c_uint32)), shape=(nnz,)).copy()
        else:
            col = np.zeros(0, dtype=np.uint32)
    finally:
        lib.synth_free(rp)
        lib.synth_free(cl)
    return row_ptr, col


def chung_lu(n: int, gamma: float, dbar: float, dmax: float, seed: int = 1, relabel: bool = True):
    """Chung-Lu graph with power-law expected degrees (exponent ``gamma``,
    mean ``dbar``, maximum ``dmax``); simple by construction."""
    return _generate(0, n, gamma, dbar, dmax, seed, relabel)


def rgg(n: int, dbar: float, seed: int = 1, relabel: bool = True):
    """2-D random geometric graph on the unit torus with mean degree ~``dbar``."""
    return _generate(1, n, 0.0, dbar, dbar, seed, relabel)


def from_edges(n: int, edges) -> tuple[np.ndarray, np.ndarray]:
    """Sorted symmetric CSR from an undirected edge list (duplicates and
    self-loops are dropped)."""
    s = set()
    for a, b in edges:
        a, b = int(a), int(b)
        if a == b:
            continue
        s.add((min(a, b), max(a, b)))
    adj = [[] for _ in range(n)]
    for a, b in s:
        adj[a].append(b)
        adj[b].append(a)
    row_ptr = np.zeros(n + 1, dtype=np.uint64)
    for i in range(n):
        row_ptr[i + 1] = row_ptr[i] + len(adj[i])
    col = np.array([x for i in range(n) for x in sorted(adj[i])], dtype=np.uint32)
    return row_ptr, col


def cycle(n: int):
    return from_edges(n, [(i, (i + 1) % n) for i in range(n)])


def complete(n: int):
    return from_edges(n, [(i, j) for i in range(n) for j in range(i + 1, n)])


def star(leaves: int):
    return from_edges(leaves + 1, [(0, i) for i in range(1, leaves + 1)])


def gnp(n: int, p: float, seed: int):
    """Small Erdos-Renyi graph for exhaustive tests (numpy generator)."""
    rng = np.random.default_rng(seed)
    e = [(i, j) for i in range(n) for j in range(i + 1, n) if rng.random() < p]
    return from_edges(n, e)


# The synthetic workloads standing in for the paper's datasets.
CONFIGS = {
    # 4-node motifs, small: n=2,000, exponent 2.5, mean degree 8, max degree 200
    "cl_n2k": dict(n=2_000, gamma=2.5, dbar=8.0, dmax=200.0, seed=1),
    # 5-node motifs at ~1M undirected edges: n=100,000, exponent 2.2, mean 20, max ~5,000
    "cl_n100k": dict(n=100_000, gamma=2.2, dbar=20.0, dmax=5_000.0, seed=1),
    # large: n=4M, exponent 2.1, mean 17, max ~20,000 (~35M edges)
    "cl_n4m": dict(n=4_000_000, gamma=2.1, dbar=17.0, dmax=20_000.0, seed=1),
}


def workload(name: str):
    c = CONFIGS[name]
    return chung_lu(c["n"], c["gamma"], c["dbar"], c["dmax"], c["seed"])
