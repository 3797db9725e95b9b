"""Algorithmic 32-byte sectors per sample -- measurement infrastructure.

For each sampled CIS, the set of distinct 32 B sectors the sampling step must
read under the device layout the library documents (include/moss.h and its
kernels): vertex alias records of 32 B (one sector, carrying the alias's
vertex record, so the drawn vertex's own 16 B record is read only when the
column keeps the draw), per-slot sigma records of 32 B (one sector, with the
alias position's pick, and for both picks the picked neighbour's list and
twin, so its vertex record is read only for a neighbour of degree 2^16 or
more), vertex records of 16 B, neighbour ids of 4 B, ACC entries of 4 B and
prefixes of squares of 8 B (Path-5 fallback); for MOSS-4Min its
vertex records of 16 B, per-slot pick records of 32 B (one sector with the
draw and both possible picks; two slot records of 32 B where the list's
total or a field is too wide) and ordered-list entries of 8 B.  Each
probe is either a lower-bound search with early exit in the shorter sorted
list (MOSS_PROBE_SEARCH, which also reads the two vertex records) or the home
bucket of the hashed edge set (MOSS_PROBE_HASH, 32 B buckets of four keys; the rare
continuation into the next bucket is not counted), or the word of the edge
filter followed by that bucket only when the filter passes (MOSS_PROBE_FILTER).
The "_filter" figures count the method's work under that layout and are the
ones the roofline uses; the "_filter_hubs" figures count what the library's
samplers read behind the filter with hub-pair bits: each of the sample's
vertices looked up in the hubs' rank table (one 8 B entry per 32 vertices),
and a pair of two hubs answered by a word of the hubs' adjacency bits instead
of the filter and the set.
The draws are replayed from the oracle's words and tables, so the
count is exact per sample; the mean over a few thousand samples is the
per-sample figure used by the roofline ("achieved" = figure x 32 B x samples
/ kernel time).

    python tests/golden/sector_model.py [workload] [samples]
writes tests/golden/sectors_<workload>.json; a workload name ending in
"_degree" is that workload renumbered as a MOSS_ORDER_DEGREE load renumbers
it (tests/helpers.degree_order).  Calls only the oracle, the shared input
generator and that test helper.
"""
from __future__ import annotations

import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import oracle  # noqa: E402
import synth  # noqa: E402

TWO64 = 1 << 64


def idx(x: int, m: int) -> int:
    return (x * m) >> 64


M64 = (1 << 64) - 1


def filter_hash(k):
    """The library's edge-filter finaliser (second xor-shift-multiply chain);
    k a Python int or a numpy uint64 array."""
    if isinstance(k, np.ndarray):
        u = np.uint64
        k = k ^ u(0x9e3779b97f4a7c15)
        k = k ^ (k >> u(31))
        k = k * u(0xbf58476d1ce4e5b9)
        k = k ^ (k >> u(27))
        k = k * u(0x94d049bb133111eb)
        return k ^ (k >> u(31))
    k ^= 0x9e3779b97f4a7c15
    k ^= k >> 31
    k = (k * 0xbf58476d1ce4e5b9) & M64
    k ^= k >> 27
    k = (k * 0x94d049bb133111eb) & M64
    return k ^ (k >> 31)


def filter_mask(h):
    if isinstance(h, np.ndarray):
        one = np.uint32(1)
        return ((one << (h & np.uint64(31)).astype(np.uint32)) | (one << ((h >> np.uint64(5)) & np.uint64(31)).astype(np.uint32))
                | (one << ((h >> np.uint64(10)) & np.uint64(31)).astype(np.uint32)))
    return (1 << (h & 31)) | (1 << ((h >> 5) & 31)) | (1 << ((h >> 10) & 31))


def edge_bucket(a: int, b: int, shift: int) -> int:
    """Home bucket of edge {a, b} in the library's hashed edge set (key
    (min << 32) | max through three xor-shift-multiply steps, top bits)."""
    k = (min(a, b) << 32) | max(a, b)
    k ^= k >> 33
    k = (k * 0xff51afd7ed558ccd) & M64
    k ^= k >> 33
    k = (k * 0xc4ceb9fe1a85ec53) & M64
    k ^= k >> 33
    return k >> shift


LEVEL_WORD = {0: 6, 1: 7, 2: 14, 3: 6}   # word of the vertex draw's level, per method


def vertex_column(vt, n, xl, xc):
    """Column of a two-level vertex table that a draw reads: the light
    level's when the level word is below its bound (or no vertex is heavy)."""
    nh = vt["nh"]
    light = nh == 0 or xl < vt["TL"]
    return (nh + idx(xc, n - nh)) if light else idx(xc, nh)


class Replay:
    def __init__(self, rp, col, probe="search", hubs=False):
        self.g = oracle.OracleGraph(rp, col)
        self.rp = rp.astype(np.int64)
        self.col = col
        self.deg = np.diff(self.rp)
        self.S = self.g.vertex()[1].astype(np.int64)
        self.seed = [self.g.vertex_table(l) for l in range(3)]
        thr, alias, acc = self.g.sigma_table()
        self.thr, self.alias, self.acc = thr.astype(np.int64), alias.astype(np.int64), acc.astype(np.int64)
        self.probe_kind = probe
        self.hubs = hubs and probe == "filter"
        buckets = 2   # the library's table: next power of two >= nnz / 2 buckets
        while buckets < (len(col) + 1) // 2:
            buckets <<= 1
        self.shift = 64 - (buckets.bit_length() - 1)
        if probe == "filter":   # the library's filter: largest power of two <= nnz / 8 words
            words = 1
            while words * 2 <= len(col) // 8:
                words <<= 1
            self.fshift = 64 - (words.bit_length() - 1)
            owner = np.repeat(np.arange(self.g.n, dtype=np.uint64), self.deg.astype(np.int64))
            c64 = col.astype(np.uint64)
            keep = owner < c64
            h = filter_hash((owner[keep] << np.uint64(32)) | c64[keep])
            self.filter = np.zeros(words, dtype=np.uint32)
            np.bitwise_or.at(self.filter, (h >> np.uint64(self.fshift)).astype(np.int64), filter_mask(h))
            if self.hubs:
                self.hub_tables()

    def hub_tables(self):
        """The library's hubs: every vertex of degree >= D, D the smallest
        degree >= 1 with at most H = min(8192, max(16, n / 16)) such
        vertices; hub i is the i-th in ascending id order."""
        n = self.g.n
        H = min(8192, max(16, n // 16))
        cnt = np.bincount(self.deg, minlength=int(self.deg.max()) + 2)
        above = np.cumsum(cnt[::-1])[::-1]          # above[d] = vertices of degree >= d
        D = next(d for d in range(1, len(above)) if above[d] <= H) if n else 1
        hubs = np.nonzero(self.deg >= D)[0] if D < len(above) else np.zeros(0, np.int64)
        self.hubs_H = H
        self.hub_index = {int(v): i for i, v in enumerate(hubs)}

    def hub_of(self, x, touched):
        """Hub index of x (or None): its rank-table entry, four 8 B entries
        (128 vertices) per sector."""
        touched.add(("hubrank", int(x) >> 7))
        return self.hub_index.get(int(x))

    def probe_all(self, pairs, verts, touched, hubs):
        """The probes of one sample; with hubs (Path-5 and MOSS-4Min under
        the filter) a pair of two hubs reads one word of the hubs' bits."""
        if not (hubs and self.hubs):
            for a, b in pairs:
                self.probe(a, b, touched)
            return
        hi = {int(z): self.hub_of(z, touched) for z in verts}
        for a, b in pairs:
            i, j = hi[int(a)], hi[int(b)]
            if i is not None and j is not None:
                touched.add(("hubbits", (i * self.hubs_H + j) >> 8))
            else:
                self.probe(a, b, touched)

    def min_tables(self):
        if not hasattr(self, "rank"):
            rl, rk, cthr, calias, gam = self.g.min_tables()
            self.rank, self.cthr_m, self.calias_m = rk.astype(np.int64), cthr, calias.astype(np.int64)
            self.gam_m = gam
            self.seed_m = self.g.vertex_table(3)

    def rank_twin(self, v, p):
        """d_{u,v} for position p (v -> u): the rank held by the twin slot."""
        u = int(self.col[p])
        ou = int(self.rp[u])
        return int(self.rank[ou + int(np.searchsorted(self.col[ou:self.rp[u + 1]], v))])

    def pick_fits(self, v, p):
        """The library reads a MOSS-4Min pick record for a list with
        Gamma-check_v < 2^32 when d_u, d_{v,u} and d_{u,v} of the position
        and of its alias position all fit 16 bits (below 0xFFFF)."""
        if int(self.gam_m[v]) >= 1 << 32:
            return False
        ap = int(self.rp[v]) + int(self.calias_m[p])
        for q in (p, ap):
            fields = (int(self.deg[int(self.col[q])]), int(self.rank[q]), self.rank_twin(v, q))
            if max(fields) >= 0xFFFF:
                return False
        return True

    def sample_min(self, seed, s, verts, cls):
        """Sectors of one MOSS-4Min sample (Algorithm 2)."""
        self.min_tables()
        t = self.touched = set()   # kept for breakdowns by table
        x = self.words(3, seed, s, 2)
        c = vertex_column(self.seed_m, self.g.n, x[6], x[0])
        t.add(("seedm", c))
        v = int(verts[0])
        if x[1] < int(self.seed_m["T"][c]):   # the column keeps the draw: its own record
            t.add(("mvert", v >> 1))
        o, d = int(self.rp[v]), int(self.deg[v])
        j = idx(x[2], d)
        if self.pick_fits(v, o + j):   # the pick record serves the whole draw
            t.add(("mpick", o + j))
            if idx(x[3], self.gam_m[v]) >= int(self.cthr_m[o + j]):
                j = int(self.calias_m[o + j])
        else:
            t.add(("mslot", o + j))
            if idx(x[3], self.gam_m[v]) >= int(self.cthr_m[o + j]):
                j = int(self.calias_m[o + j])
                t.add(("mslot", o + j))
        u = int(self.col[o + j])
        dvu = int(self.rank[o + j])
        ou = int(self.rp[u])
        duv = self.rank_twin(v, o + j)
        t.add(("rlist", (o + idx(x[4], dvu)) >> 2))
        t.add(("rlist", (ou + idx(x[5], duv)) >> 2))
        w, r = int(verts[2]), int(verts[3])
        if cls:
            if self.probe_kind == "search":
                t.add(("vert", w >> 1))
                t.add(("vert", r >> 1))
            self.probe_all(((v, r), (u, w), (w, r)), (v, u, w, r), t, True)
        return len(t)

    def words(self, method, seed, s, blocks):
        return oracle.sample_words(method, seed, s, 4 * blocks)

    def probe(self, a, b, touched):
        if self.probe_kind == "filter":   # filter word (8 per sector); the set only when it may hold the pair
            a, b = int(a), int(b)
            h = filter_hash((min(a, b) << 32) | max(a, b))
            w = h >> self.fshift
            touched.add(("filter", w >> 3))
            m = filter_mask(h)
            if int(self.filter[w]) & m == m:
                touched.add(("hash", edge_bucket(a, b, self.shift)))
            return
        if self.probe_kind == "hash":   # home bucket: one 32 B sector
            touched.add(("hash", edge_bucket(int(a), int(b), self.shift)))
            return
        da, db = self.deg[a], self.deg[b]
        if da <= db:
            lo, ln, key = self.rp[a], da, b
        else:
            lo, ln, key = self.rp[b], db, a
        while ln > 0:
            half = ln >> 1
            p = lo + half
            touched.add(("col", int(p) >> 3))
            val = int(self.col[p])
            if val == key:
                return
            if val < key:
                lo, ln = p + 1, ln - half - 1
            else:
                ln = half

    def hub(self, x, touched):
        """The slot record carries a picked neighbour's list and twin; only a
        neighbour with 2^16 or more neighbours needs its vertex record."""
        if int(self.deg[x]) >= 1 << 16:
            touched.add(("vert", x >> 1))

    def sigma(self, v, xc, xt, touched):
        """One sigma draw: the 32 B slot record (the column's pick and its
        alias's)."""
        o, d, S = int(self.rp[v]), int(self.deg[v]), int(self.S[v])
        j = idx(xc, d)
        touched.add(("slot", o + j))
        if idx(xt, S) < int(self.thr[o + j]):
            return j
        return int(self.alias[o + j])

    def fallback(self, v, x12, x13, touched):
        """The Path-5 fallback as the kernel runs it: tau by binary search
        over S ACC - sq, mu by binary search over ACC with u's interval removed."""
        o, d, S = int(self.rp[v]), int(self.deg[v]), int(self.S[v])
        acc = [int(a) for a in self.acc[o:o + d]]
        w = [(acc[i + 1] if i + 1 < d else S) - acc[i] for i in range(d)]
        sq = [0] * d
        for i in range(1, d):
            sq[i] = sq[i - 1] + w[i - 1] ** 2
        touched.add(("acc", (o + d - 1) >> 3))
        touched.add(("sq", (o + d - 1) >> 2))
        G = S * S - (sq[d - 1] + w[d - 1] ** 2)
        y = idx(x12, G)
        lo, ln = 0, d
        while ln > 0:
            half = ln >> 1
            p = lo + half
            touched.add(("acc", (o + p) >> 3))
            touched.add(("sq", (o + p) >> 2))
            if S * acc[p] - sq[p] <= y:
                lo, ln = p + 1, ln - half - 1
            else:
                ln = half
        iu = lo - 1
        touched.add(("acc", (o + iu) >> 3))
        if iu + 1 < d:
            touched.add(("acc", (o + iu + 1) >> 3))
        y2 = idx(x13, S - w[iu])
        if y2 >= acc[iu]:
            y2 += w[iu]
        lo, ln = 0, d
        while ln > 0:
            half = ln >> 1
            touched.add(("acc", (o + lo + half) >> 3))
            if acc[lo + half] <= y2:
                lo, ln = lo + half + 1, ln - half - 1
            else:
                ln = half
        return iu, lo - 1

    def sample(self, method, seed, s, verts, cls):
        t = self.touched = set()   # kept for breakdowns by table
        vt = self.seed[method]
        x = self.words(method, seed, s, 4)
        c = vertex_column(vt, self.g.n, x[LEVEL_WORD[method]], x[0])
        t.add(("seed", c))
        v = int(verts[0])
        if x[1] < int(vt["T"][c]):   # the column keeps the draw: its own vertex record
            t.add(("vert", v >> 1))
        o = int(self.rp[v])
        if method == 2:
            iu = self.sigma(v, x[4], x[5], t)
            iw = self.sigma(v, x[6], x[7], t)
            if iu == iw:
                iu = self.sigma(v, x[8], x[9], t)
                iw = self.sigma(v, x[10], x[11], t)
                if iu == iw:  # fallback: two binary searches and two slot records
                    iu, iw = self.fallback(v, x[12], x[13], t)
                    # the binary searches land where the oracle's scan did
                    assert int(self.col[o + iu]) == int(verts[1]) and int(self.col[o + iw]) == int(verts[2])
                    t.add(("slot", o + iu))
                    t.add(("slot", o + iw))
            u, w, r, tt = (int(z) for z in verts[1:5])
            self.hub(u, t)
            self.hub(w, t)
            ju = int(np.searchsorted(self.col[self.rp[u]:self.rp[u + 1]], r))
            jt = int(np.searchsorted(self.col[self.rp[w]:self.rp[w + 1]], tt))
            t.add(("col", (int(self.rp[u]) + ju) >> 3))
            t.add(("col", (int(self.rp[w]) + jt) >> 3))
            if cls:
                if self.probe_kind == "search":
                    t.add(("vert", r >> 1))
                    t.add(("vert", tt >> 1))
                self.probe_all(((v, r), (v, tt), (u, w), (u, tt), (w, r), (r, tt)), (v, u, w, r, tt), t, True)
            return len(t)
        iu = self.sigma(v, x[2], x[3], t)
        u, w, r = int(verts[1]), int(verts[2]), int(verts[3])
        col_v = self.col[o:o + int(self.deg[v])]
        t.add(("col", (o + int(np.searchsorted(col_v, w))) >> 3))
        self.hub(u, t)
        if method == 0:
            ju = int(np.searchsorted(self.col[self.rp[u]:self.rp[u + 1]], r))
            t.add(("col", (int(self.rp[u]) + ju) >> 3))
            if cls:
                if self.probe_kind == "search":
                    t.add(("vert", w >> 1))
                    t.add(("vert", r >> 1))
                self.probe_all(((v, r), (u, w), (w, r)), (v, u, w, r), t, True)
            return len(t)
        tt = int(verts[4])
        t.add(("col", (o + int(np.searchsorted(col_v, r))) >> 3))
        jt = int(np.searchsorted(self.col[self.rp[u]:self.rp[u + 1]], tt))
        t.add(("col", (int(self.rp[u]) + jt) >> 3))
        if cls:
            if self.probe_kind == "search":
                for z in (w, r, tt):
                    t.add(("vert", z >> 1))
            self.probe_all(((u, w), (u, r), (w, r), (v, tt), (w, tt), (r, tt)), (v, u, w, r, tt), t, True)
        return len(t)


def model(workload: str, samples: int = 4000, seed: int = 42) -> dict:
    if workload.endswith("_degree"):
        sys.path.insert(0, os.path.join(ROOT, "tests"))
        from helpers import degree_order
        _, rp, col = degree_order(*synth.workload(workload[: -len("_degree")]))
    else:
        rp, col = synth.workload(workload)
    out = {"workload": workload, "samples": samples, "seed": seed,
           "layout": ("32 B vertex alias records with the alias's vertex record, 32 B slot records with the "
                      "alias's pick and both picks' neighbour list and twin, 16 B vertex records, "
                      "4 B ids and ACC, 8 B Q, 32 B edge-hash buckets (home bucket counted), 4 B edge-filter words "
                      "(the set's bucket only when the filter passes); MOSS-4Min: 16 B "
                      "vertex, 32 B pick (32 B slot where too wide), 8 B list records; _filter_hubs adds 8 B "
                      "hub-map slots and 4 B hub-bit words; 32 B sectors"),
           "source": "written by tests/golden/sector_model.py"}
    for probe, suffix in (("search", "_search"), ("hash", "_hash"), ("filter", "_filter"), ("hubs", "_filter_hubs")):
        rep = Replay(rp, col, "filter" if probe == "hubs" else probe, hubs=probe == "hubs")
        for method, name in ((0, "MOSS4"), (1, "T5"), (2, "PATH5")):
            first = 1_000_000
            _, cls, verts = rep.g.run(method, seed, samples, first=first, record=True)
            n = [rep.sample(method, seed, first + i, verts[i], int(cls[i])) for i in range(samples)]
            out[name + suffix] = {"sectors_per_sample": float(np.mean(n)),
                                  "stderr": float(np.std(n) / np.sqrt(samples)),
                                  "collision_rate": float(np.mean(cls == 0))}
        first = 1_000_000
        _, cls, verts = rep.g.run(oracle.MOSS4MIN, seed, samples, first=first, record=True)
        n = [rep.sample_min(seed, first + i, verts[i], int(cls[i])) for i in range(samples)]
        out["MOSS4MIN" + suffix] = {"sectors_per_sample": float(np.mean(n)),
                                    "stderr": float(np.std(n) / np.sqrt(samples)),
                                    "collision_rate": float(np.mean(cls == 0))}
    return out


if __name__ == "__main__":
    wl = sys.argv[1] if len(sys.argv) > 1 else "cl_n100k"
    ns = int(sys.argv[2]) if len(sys.argv) > 2 else 4000
    res = model(wl, ns)
    path = os.path.join(ROOT, "tests", "golden", f"sectors_{wl}.json")
    with open(path, "w") as f:
        json.dump(res, f, indent=1)
        f.write("\n")
    print(json.dumps(res, indent=1))
