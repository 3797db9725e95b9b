"""Independent test helpers: motif identification with networkx, brute-force
subgraph enumeration and the paper's printed phi tables (tests/golden)."""
from __future__ import annotations

import itertools
import os
from functools import lru_cache

import networkx as nx
import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _read_table(name: str) -> dict[int, tuple[int, ...]]:
    out = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            vals = [int(x) for x in line.split()]
            out[vals[0]] = tuple(vals[1:])
    return out


def table2() -> dict[int, tuple[int, int, int]]:
    """Table 2: class -> (phi1 forks, phi2 5-paths, phi3 4-stars)."""
    return _read_table("table2_phi5.txt")


def phi4() -> dict[int, tuple[int, int]]:
    """Sec. 4.1.2: class -> (phi1 3-paths, phi2 3-stars)."""
    return _read_table("phi4.txt")


def _count_copies(H: nx.Graph, P: nx.Graph) -> int:
    """Number of (not necessarily induced) subgraphs of H isomorphic to P."""
    mono = sum(1 for _ in nx.algorithms.isomorphism.GraphMatcher(H, P).subgraph_monomorphisms_iter())
    aut = sum(1 for _ in nx.algorithms.isomorphism.GraphMatcher(P, P).isomorphisms_iter())
    assert mono % aut == 0
    return mono // aut


def _patterns(k: int):
    if k == 4:
        return [nx.path_graph(4), nx.star_graph(3)]
    fork = nx.Graph([(0, 1), (0, 2), (0, 3), (1, 4)])
    return [fork, nx.path_graph(5), nx.star_graph(4)]


@lru_cache(maxsize=None)
def motif_atlas(k: int):
    """[(graph, signature, class)] for every connected graph on k vertices;
    the class is the row of the paper's table carrying that signature."""
    table = phi4() if k == 4 else table2()
    by_sig = {v: i for i, v in table.items()}
    out = []
    for H in nx.graph_atlas_g():
        if H.number_of_nodes() != k or not nx.is_connected(H):
            continue
        sig = tuple(_count_copies(H, P) for P in _patterns(k))
        out.append((H, sig, by_sig.get(sig)))
    return out


def nx_class(k: int, edges) -> int:
    """Class of the graph on vertices 0..k-1 with the given edges (0 if
    disconnected), identified by isomorphism against the atlas."""
    G = nx.Graph()
    G.add_nodes_from(range(k))
    G.add_edges_from(edges)
    if not nx.is_connected(G):
        return 0
    for H, _sig, cls in motif_atlas(k):
        if H.number_of_edges() == G.number_of_edges() and nx.is_isomorphic(G, H):
            return cls
    raise AssertionError("no atlas match")


@lru_cache(maxsize=None)
def mask_classes(k: int) -> tuple[int, ...]:
    pairs = [(i, j) for i in range(k) for j in range(i + 1, k)]
    out = []
    for mask in range(1 << len(pairs)):
        out.append(nx_class(k, [pairs[b] for b in range(len(pairs)) if mask >> b & 1]))
    return tuple(out)


def adjacency_sets(row_ptr, col):
    n = len(row_ptr) - 1
    return [set(int(x) for x in col[int(row_ptr[v]):int(row_ptr[v + 1])]) for v in range(n)]


def induced_class(adj, verts) -> int:
    """Class of the subgraph induced by verts (ordered), via the mask table."""
    k = len(verts)
    mask = 0
    b = 0
    for i in range(k):
        for j in range(i + 1, k):
            if verts[j] in adj[verts[i]]:
                mask |= 1 << b
            b += 1
    return mask_classes(k)[mask]


def brute_force_cis(row_ptr, col, k: int) -> dict[frozenset, int]:
    """Every connected induced k-subgraph (as a vertex set) with its class,
    by scanning all k-subsets (tiny graphs only)."""
    adj = adjacency_sets(row_ptr, col)
    n = len(adj)
    out = {}
    for vs in itertools.combinations(range(n), k):
        c = induced_class(adj, vs)
        if c:
            out[frozenset(vs)] = c
    return out


def class_counts(cis: dict, nclass: int) -> np.ndarray:
    c = np.zeros(22, dtype=np.int64)
    for cls in cis.values():
        c[cls] += 1
    return c


SLOT_HUB = 0xFFFFFFFF


def slot_twin(slot: np.ndarray) -> np.ndarray:
    """Twin (position of v in N_col) of exported 32-byte slot records: the low
    16 bits of word 1, or word 4 for a neighbour of degree 2^16 or more."""
    nb = slot[:, 1].astype(np.int64)
    return np.where(nb == SLOT_HUB, slot[:, 4].astype(np.int64), nb & 0xFFFF)


def expected_slot_neighbour(rp: np.ndarray, col: np.ndarray, twin: np.ndarray):
    """Words 1 and 4 of the slot records that the library's layout defines
    for neighbour lists (rp, col) and twins: (twin | d_x << 16, off_x), or
    (SLOT_HUB, twin) when d_x >= 2^16."""
    c64 = col.astype(np.int64)
    rp64 = rp.astype(np.int64)
    dx = rp64[c64 + 1] - rp64[c64]
    hub = dx >= 1 << 16
    nb = np.where(hub, SLOT_HUB, twin | (dx << 16))
    off = np.where(hub, twin, rp64[c64])
    return nb.astype(np.uint32), off.astype(np.uint32)


def oracle_counts(og, method: int, seed: int, first: int, count: int, threads: int | None = None,
                  rng: int = 0) -> np.ndarray:
    """The oracle's counts of samples [first, first + count) of one method,
    split into id chunks run on all host cores.  The oracle's sampler only
    reads its tables and ctypes releases the GIL around it, so threads share
    one oracle graph; integer counts add up the same in any order."""
    import concurrent.futures as cf
    threads = threads or os.cpu_count() or 1
    chunk = max(1 << 16, -(-count // (8 * threads)))
    parts = [(a, min(chunk, first + count - a)) for a in range(first, first + count, chunk)]
    total = np.zeros(22, dtype=np.uint64)
    if not parts:
        return total
    with cf.ThreadPoolExecutor(max_workers=threads) as ex:
        for c in ex.map(lambda p: og.run(method, seed, p[1], first=p[0], rng=rng), parts):
            total += c
    return total


def close_estimates(r, o, og, k):
    """A library result r against the oracle's finalize o: estimates,
    variances and concentrations within 1e-9 relative (the class closed by
    an identity, n_2 or eta_2, relative to Lambda_3 or Lambda_4), the
    triangle estimate (k = 4) and the mix weights (k = 5)."""
    n = 7 if k == 4 else 22
    lam = float(og.Lambda3 if k == 4 else og.Lambda4)
    for i in range(1, n):
        if i == 2:
            assert abs(r["est"][i] - o["est"][i]) <= 1e-9 * max(lam, 1.0), (k, i)
            assert abs(r["var"][i] - o["var"][i]) <= 1e-9 * max(abs(o["var"][i]), 1.0) + 1e-9 * lam ** 2 / 1e6
            continue
        assert abs(r["est"][i] - o["est"][i]) <= 1e-9 * max(abs(o["est"][i]), 1e-300), (k, i, r["est"][i], o["est"][i])
        assert abs(r["var"][i] - o["var"][i]) <= 1e-9 * max(abs(o["var"][i]), 1e-300), (k, i)
    for i in range(1, n):
        assert abs(r["conc"][i] - o["conc"][i]) <= 1e-9 * max(abs(o["conc"][i]), 1e-300) + 1e-12, (k, i)
    if k == 4:
        assert abs(r["triangles"] - o["triangles"]) <= 1e-9 * max(abs(o["triangles"]), 1e-300)
    else:
        for i in range(1, n):
            for l in range(2):
                assert abs(r["lam"][l][i] - o["lam"][l][i]) <= 1e-9


def order_key(deg) -> np.ndarray:
    """Degree key of MOSS_ORDER_DEGREE: d below 16, else quarter-octave
    classes 16 + 4 (L - 5) + the two bits below the leading one (L = bit
    length of d)."""
    d = np.asarray(deg, dtype=np.int64)
    L = np.zeros_like(d)
    nz = d > 0
    L[nz] = np.floor(np.log2(d[nz])).astype(np.int64) + 1
    # exact bit length (the float log can be off by one next to a power of two)
    L[nz & ((1 << np.maximum(L - 1, 0)) > d)] -= 1
    L[nz & ((1 << L) <= d)] += 1
    sh = np.maximum(L - 3, 0)
    return np.where(d < 16, d, 16 + 4 * (L - 5) + ((d >> sh) & 3))


def degree_order(rp, col):
    """The graph renumbered as a MOSS_ORDER_DEGREE load does: internal vertex
    i is input vertex order[i], sorted by key descending, then input id;
    returns (order, row_ptr, col) of the renumbered graph, lists ascending."""
    rp = np.asarray(rp, dtype=np.int64)
    col = np.asarray(col, dtype=np.int64)
    n = len(rp) - 1
    deg = np.diff(rp)
    order = np.argsort(-order_key(deg), kind="stable")
    inv = np.empty(n, dtype=np.int64)
    inv[order] = np.arange(n)
    nrp = np.zeros(n + 1, dtype=np.uint64)
    nrp[1:] = np.cumsum(deg[order])
    nrow = inv[np.repeat(np.arange(n), deg)]
    ncol = inv[col]
    idx = np.lexsort((ncol, nrow))
    return order.astype(np.uint32), nrp, ncol[idx].astype(np.uint32)
