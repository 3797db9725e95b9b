"""Exact sampling distributions of the oracle's samplers (CPU).

The oracle's per-sample function is driven with chosen random words.  Every
draw maps a 64-bit word x to an outcome through floor(x m / 2^64) or a
threshold test, so the exact probability of each outcome is an integer count
of words over 2^64.  Enumerating every branch of every draw and weighting the
oracle's resulting CIS by the product of those counts gives the oracle's exact
distribution, which is compared with the sampling-weight theorems:

* Theorem 2 (MOSS-4):  P(s) = 2 phi^(1)_i / Gamma        for s in C_i^(4)
* Theorem 6 (T-5):     P(s) = 2 phi^(1)_i / Gamma^(1)    for s in C_i^(5)
* Theorem 8 (Path-5):  P(s) = 2 phi^(2)_i / Gamma^(2)    for s in C_i^(5)
  and, inside Path-5, P(u, w | v) = tau_u mu_w = (d_u-1)(d_w-1)/Gamma^(2)_v.

The CIS sets and their classes come from brute force over all k-subsets with
networkx isomorphism (tests/helpers.py), the phi values from the paper's
printed tables (tests/golden).  The only deviation allowed is the 2^-64
quantisation of each draw.  The vertex draw has three words (level, column,
threshold); each test runs with one level (the default below 2^20
vertices), at split 20 (every tiny graph's vertices are then heavy) and at
split 2, where at most four vertices are heavy and both levels are drawn.
"""
from __future__ import annotations

from collections import defaultdict
from fractions import Fraction

import numpy as np
import pytest

import oracle
import synth
from helpers import adjacency_sets, brute_force_cis, phi4, table2

TWO64 = 1 << 64


def cdiv(a: int, b: int) -> int:
    return -(-a // b)


def iw(j: int, m: int) -> int:
    """Smallest word x with floor(x m / 2^64) = j (2^64 for j = m)."""
    return cdiv(j * TWO64, m)


def ic(j: int, m: int) -> int:
    """Number of words x with floor(x m / 2^64) = j."""
    return iw(j + 1, m) - iw(j, m)


def ic_range(a: int, b: int, m: int) -> int:
    """Number of words x with floor(x m / 2^64) in [a, b)."""
    return iw(b, m) - iw(a, m)


def triangles(adj) -> int:
    n = len(adj)
    return sum(1 for a in range(n) for b in adj[a] if b > a for c in adj[b] if c > b and c in adj[a])


LEVEL_WORD = {0: 6, 1: 7, 2: 14, 3: 6}   # index of the vertex draw's level word per method
SPLITS = [oracle.ONE_LEVEL, oracle.VSPLIT, 2]


def put_level(words, method, xl):
    """words with the level word of the vertex draw set to xl."""
    w = list(words) + [0] * (16 - len(words))
    w[LEVEL_WORD[method]] = xl
    return w


class Tables:
    def __init__(self, rp, col, which, vsplit=None):
        self.g = oracle.OracleGraph(rp, col, vsplit=vsplit)
        self.rp = [int(x) for x in rp]
        self.col = [int(x) for x in col]
        self.n = len(rp) - 1
        self.deg = [self.rp[v + 1] - self.rp[v] for v in range(self.n)]
        self.S = [sum(self.deg[x] - 1 for x in self.col[self.rp[v]:self.rp[v + 1]]) for v in range(self.n)]
        vt = self.g.vertex_table(which)
        self.nh, self.TL = vt["nh"], vt["TL"]
        self.self_ = [int(x) for x in vt["self"]]
        self.T = [int(x) for x in vt["T"]]
        self.alias = [int(x) for x in vt["alias"]]
        thr, galias, acc = self.g.sigma_table()
        self.thr = [int(x) for x in thr]
        self.galias = [int(x) for x in galias]
        self.acc = [int(x) for x in acc]

    def seed_branches(self):
        """(count over 2^192, x_level, x0, x1, v) for every seed-draw branch:
        the light level for level words below TL (always, without heavy
        vertices), the heavy one above; then column and threshold."""
        levels = []
        if self.nh == 0:
            levels.append((TWO64, 0, 0, self.n))
        else:
            if self.TL > 0:
                levels.append((self.TL, 0, self.nh, self.n - self.nh))
            levels.append((TWO64 - self.TL, TWO64 - 1, 0, self.nh))
        for cl, xl, base, m in levels:
            for c in range(m):
                cc = ic(c, m)
                t = self.T[base + c]
                if t > 0:
                    yield cl * cc * t, xl, iw(c, m), 0, self.self_[base + c]
                if TWO64 - t > 0:
                    yield cl * cc * (TWO64 - t), xl, iw(c, m), TWO64 - 1, self.alias[base + c]

    def sigma_branches(self, v):
        """(count over 2^128, xc, xt, position) for every sigma-draw branch."""
        o, d, S = self.rp[v], self.deg[v], self.S[v]
        for j in range(d):
            cj = ic(j, d)
            keep = iw(self.thr[o + j], S)
            if keep > 0:
                yield cj * keep, iw(j, d), 0, j
            if TWO64 - keep > 0:
                yield cj * (TWO64 - keep), iw(j, d), TWO64 - 1, self.galias[o + j]


def check_against_theorem(probs, denom_bits, cis, phi_of, Gamma, extra=None):
    total = sum(probs.values())
    assert total == 1 << denom_bits, "branch probabilities do not sum to one"
    for s, cls in cis.items():
        ideal = Fraction(2 * phi_of(cls), Gamma)
        got = Fraction(probs.get(s, 0), 1 << denom_bits)
        if ideal == 0:
            assert got == 0, (s, cls)
        else:
            assert abs(got - ideal) <= ideal * Fraction(1, 10 ** 12), (s, cls, float(got), float(ideal))
    for s in probs:
        if s != "miss":
            assert s in cis, s
    if extra is not None:
        ideal = extra
        got = Fraction(probs.get("miss", 0), 1 << denom_bits)
        assert abs(got - ideal) <= max(ideal, Fraction(1, 10 ** 30)) * Fraction(1, 10 ** 12)


def tiny_graphs():
    out = [synth.gnp(7, 0.55, s) for s in (3, 11, 19)]
    out.append(synth.from_edges(7, [(0, 1), (1, 2), (2, 3), (3, 0), (0, 2), (2, 4), (4, 5), (5, 6), (6, 4), (1, 5)]))
    return out


@pytest.mark.parametrize("vsplit", SPLITS)
@pytest.mark.parametrize("gi", range(4))
def test_moss4_distribution_is_theorem2(gi, vsplit):
    rp, col = tiny_graphs()[gi]
    t = Tables(rp, col, 0, vsplit)
    g = t.g
    if g.Gamma[0] == 0:
        pytest.skip("no 3-path")
    probs = defaultdict(int)
    for c0, xl, x0, x1, v in t.seed_branches():
        dv = t.deg[v]
        assert dv >= 2 and t.S[v] > 0, "zero-weight vertex drawn"
        for c1, x2, x3, iu in t.sigma_branches(v):
            u = t.col[t.rp[v] + iu]
            du = t.deg[u]
            for jw in range(dv - 1):
                for jr in range(du - 1):
                    verts, cls = g.sample_words(oracle.MOSS4, put_level([x0, x1, x2, x3, iw(jw, dv - 1),
                                                                         iw(jr, du - 1)], 0, xl))
                    assert verts[0] == v and verts[1] == u
                    key = frozenset(verts[:4]) if cls else "miss"
                    probs[key] += c0 * c1 * ic(jw, dv - 1) * ic(jr, du - 1)
    cis = brute_force_cis(rp, col, 4)
    p4 = phi4()
    adj = adjacency_sets(rp, col)
    # r = w closes a triangle: 6 ordered draws of probability 1/Gamma each
    check_against_theorem(probs, 64 * 7, cis, lambda c: p4[c][0], g.Gamma[0],
                          extra=Fraction(6 * triangles(adj), g.Gamma[0]))


@pytest.mark.parametrize("vsplit", SPLITS)
@pytest.mark.parametrize("gi", range(4))
def test_t5_distribution_is_theorem6(gi, vsplit):
    rp, col = tiny_graphs()[gi]
    t = Tables(rp, col, 1, vsplit)
    g = t.g
    if g.Gamma[1] == 0:
        pytest.skip("no fork")
    probs = defaultdict(int)
    for c0, xl, x0, x1, v in t.seed_branches():
        dv = t.deg[v]
        assert dv >= 3
        for c1, x2, x3, iu in t.sigma_branches(v):
            u = t.col[t.rp[v] + iu]
            du = t.deg[u]
            for jw in range(dv - 1):
                for jr in range(dv - 2):
                    for jt in range(du - 1):
                        words = [x0, x1, x2, x3, iw(jw, dv - 1), iw(jr, dv - 2), iw(jt, du - 1)]
                        verts, cls = g.sample_words(oracle.T5, put_level(words, 1, xl))
                        key = frozenset(verts) if cls else "miss"
                        probs[key] += c0 * c1 * ic(jw, dv - 1) * ic(jr, dv - 2) * ic(jt, du - 1)
    cis = brute_force_cis(rp, col, 5)
    t2 = table2()
    check_against_theorem(probs, 64 * 8, cis, lambda c: t2[c][0], g.Gamma[1])


def pair_branches(t: Tables, v: int):
    """All branches of the Path-5 (u, w) draw of vertex v as
    (count over 2^(64*10), words[4..13], iu, iw).  The branch structure is the
    oracle's documented schedule: two sigma x sigma attempts, then tau / mu."""
    o, d, S = t.rp[v], t.deg[v], t.S[v]
    w_ = [t.deg[x] - 1 for x in t.col[o:o + d]]
    out = []

    def fallback(prefix_count, prefix_words):
        G = S * S - sum(x * x for x in w_)
        run = 0
        for iu_ in range(d):
            tw = w_[iu_] * (S - w_[iu_])
            if tw == 0:
                run += tw
                continue
            cu = ic_range(run, run + tw, G)
            xu = iw(run, G)
            run += tw
            M = S - w_[iu_]
            for iw_ in range(d):
                if iw_ == iu_ or w_[iw_] == 0:
                    continue
                lo = t.acc[o + iw_] if iw_ < iu_ else t.acc[o + iw_] - w_[iu_]
                cw = ic_range(lo, lo + w_[iw_], M)
                out.append((prefix_count * cu * cw, prefix_words + [xu, iw(lo, M)], iu_, iw_))

    for ca, xa, xb, iua in t.sigma_branches(v):
        for cb, xc, xd, iwa in t.sigma_branches(v):
            if iua != iwa:
                out.append((ca * cb * TWO64 ** 6, [xa, xb, xc, xd, 0, 0, 0, 0, 0, 0], iua, iwa))
                continue
            for cc_, xe, xf, iub in t.sigma_branches(v):
                for cd, xg, xh, iwb in t.sigma_branches(v):
                    if iub != iwb:
                        out.append((ca * cb * cc_ * cd * TWO64 ** 2, [xa, xb, xc, xd, xe, xf, xg, xh, 0, 0], iub, iwb))
                    else:
                        fallback(ca * cb * cc_ * cd, [xa, xb, xc, xd, xe, xf, xg, xh])
    return out


@pytest.mark.parametrize("vsplit", SPLITS)
@pytest.mark.parametrize("gi", range(4))
def test_path5_distribution_is_theorem8(gi, vsplit):
    rp, col = tiny_graphs()[gi]
    t = Tables(rp, col, 2, vsplit)
    g = t.g
    if g.Gamma[2] == 0:
        pytest.skip("no 5-path")
    probs = defaultdict(int)
    for c0, xl, x0, x1, v in t.seed_branches():
        o = t.rp[v]
        pairs = defaultdict(int)
        rep = {}
        for cnt, words, iu_, iw_ in pair_branches(t, v):
            verts, _cls = g.sample_words(oracle.PATH5, put_level([x0, x1, 0, 0] + words, 2, xl))
            assert verts[0] == v
            assert (verts[1], verts[2]) == (t.col[o + iu_], t.col[o + iw_])
            pairs[(iu_, iw_)] += cnt
            rep[(iu_, iw_)] = words
        # P(u, w | v) = tau_u mu_w = (d_u - 1)(d_w - 1) / Gamma^(2)_v  (Sec. 5.1.2)
        G2v = t.S[v] ** 2 - sum((t.deg[x] - 1) ** 2 for x in t.col[o:o + t.deg[v]])
        assert sum(pairs.values()) == TWO64 ** 10
        for (iu_, iw_), cnt in pairs.items():
            ideal = Fraction((t.deg[t.col[o + iu_]] - 1) * (t.deg[t.col[o + iw_]] - 1), G2v)
            assert abs(Fraction(cnt, TWO64 ** 10) - ideal) <= ideal * Fraction(1, 10 ** 12)
        for (iu_, iw_), cnt in pairs.items():
            u, w = t.col[o + iu_], t.col[o + iw_]
            du, dw = t.deg[u], t.deg[w]
            for jr in range(du - 1):
                for jt in range(dw - 1):
                    verts, cls = g.sample_words(oracle.PATH5, put_level([x0, x1, iw(jr, du - 1), iw(jt, dw - 1)]
                                                                         + rep[(iu_, iw_)], 2, xl))
                    key = frozenset(verts) if cls else "miss"
                    probs[key] += c0 * cnt * ic(jr, du - 1) * ic(jt, dw - 1)
    cis = brute_force_cis(rp, col, 5)
    t2 = table2()
    check_against_theorem(probs, 64 * 15, cis, lambda c: t2[c][1], g.Gamma[2])


def test_path5_fallback_branch_is_reached():
    """A vertex whose neighbourhood weight sits on one neighbour makes both
    sigma x sigma attempts collide often; its pair law must still be exact."""
    # v=0 has neighbours 1 (degree 6) and 2 (degree 2)
    edges = [(0, 1), (0, 2), (2, 3)] + [(1, j) for j in range(4, 9)]
    rp, col = synth.from_edges(9, edges)
    t = Tables(rp, col, 2)
    br = pair_branches(t, 0)
    fb = [b for b in br if b[1][8] != 0 or b[1][9] != 0]
    assert fb, "fallback never taken"
    tot = defaultdict(int)
    for cnt, words, iu_, iw_ in br:
        verts, _ = t.g.sample_words(oracle.PATH5, [iw(0, 9), 0, 0, 0] + words)
        tot[(verts[1], verts[2])] += cnt
    d = [t.deg[x] - 1 for x in t.col[0:2]]
    G = (d[0] + d[1]) ** 2 - d[0] ** 2 - d[1] ** 2
    assert abs(Fraction(tot[(1, 2)], TWO64 ** 10) - Fraction(d[0] * d[1], G)) < Fraction(1, 10 ** 12)
    assert abs(Fraction(tot[(2, 1)], TWO64 ** 10) - Fraction(d[0] * d[1], G)) < Fraction(1, 10 ** 12)
