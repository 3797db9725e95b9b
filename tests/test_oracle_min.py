"""Pins of the oracle's MOSS-4Min (Sec. 4.2, Algorithm 2) on the CPU.

Algorithm 2 draws an ordered tuple (v, u, w, r) -- v from pi-check, u from
sigma-check^(v) (eq. 3), w uniform in N_{v,u}, r uniform in N_{u,v} -- and
every admissible tuple has probability
  Gamma-check_v / Gamma-check * d_{u,v} d_{v,u} / Gamma-check_v
  * 1 / d_{v,u} * 1 / d_{u,v} = 1 / Gamma-check,
so Gamma-check equals the number of admissible tuples and a CIS is drawn with
probability (tuples onto it) / Gamma-check.  The tests below

* recompute the total order, N_{u,v}, d_{u,v} and Gamma-check_v by brute force
  from their definitions (Sec. 3.2, Sec. 4.2) and compare the oracle's tables;
* enumerate every branch of every random word, as in test_oracle_exact, and
  compare the oracle's exact distribution with the brute-force tuple counts;
* check that the c(s) the oracle reports is half the number of tuples onto s
  (a path is drawn from both of its orientations), that it is 1 for every
  4-cycle and 3 for every 4-clique (Theorem 4), and that a diamond whose degree-2
  vertices outrank its chord has c = 3 (Theorem 4 says 1 for every diamond);
* check the estimator of the finalize step is exactly unbiased under the exact
  distribution, and its variance and the Theorem 1 mix with MOSS-4 against
  repeated sampling;
* check the closed forms Gamma-check(K_n) = 6 C(n,4) + 2 C(n,3) (every 4-set a
  clique with c = 3, plus the r = w tuples (v, u, w) with w above both),
  Gamma-check(C_4) = 2 and Gamma-check(star) = 0.
"""
from __future__ import annotations

import itertools
import math
from collections import defaultdict
from fractions import Fraction

import numpy as np
import pytest

import oracle
import synth
from helpers import adjacency_sets, brute_force_cis

TWO64 = 1 << 64
Z = 4.5


def cdiv(a: int, b: int) -> int:
    return -(-a // b)


def iw(j: int, m: int) -> int:
    return cdiv(j * TWO64, m)


def ic(j: int, m: int) -> int:
    return iw(j + 1, m) - iw(j, m)


class Brute:
    """The definitions of Sec. 3.2 and Sec. 4.2, evaluated naively."""

    def __init__(self, rp, col):
        self.adj = adjacency_sets(rp, col)
        self.n = len(self.adj)
        self.deg = [len(a) for a in self.adj]

    def above(self, a: int, b: int) -> bool:
        """a > b in the total order: higher degree, ties broken by the larger id."""
        return self.deg[a] > self.deg[b] or (self.deg[a] == self.deg[b] and a > b)

    def N(self, u: int, v: int):
        """N_{u,v}: neighbours of u above v."""
        return sorted(x for x in self.adj[u] if self.above(x, v))

    def gamma_v(self, v: int) -> int:
        return sum(len(self.N(v, x)) * len(self.N(x, v)) for x in self.adj[v])

    def tuples(self):
        """Every admissible (v, u, w, r) of Algorithm 2."""
        for v in range(self.n):
            for u in self.adj[v]:
                for w in self.N(v, u):
                    for r in self.N(u, v):
                        yield v, u, w, r


def tiny_graphs():
    out = [synth.gnp(8, 0.55, s) for s in (3, 11, 19)]
    out.append(synth.from_edges(7, [(0, 1), (1, 2), (2, 3), (3, 0), (0, 2), (2, 4), (4, 5), (5, 6), (6, 4), (1, 5)]))
    out.append(decorated_diamond())
    return out


def decorated_diamond():
    """Diamond 0-1 chord, 2 and 3 of degree 2 inside it, each given two pendant
    vertices so that 2 and 3 outrank 0 and 1 in the total order."""
    return synth.from_edges(8, [(0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 4), (2, 5), (3, 6), (3, 7)])


@pytest.mark.parametrize("gi", range(5))
def test_tables_match_definitions(gi):
    rp, col = tiny_graphs()[gi]
    b = Brute(rp, col)
    g = oracle.OracleGraph(rp, col)
    rl, rk, cthr, calias, gam = g.min_tables()
    rp = [int(x) for x in rp]
    col = [int(x) for x in col]
    for v in range(b.n):
        o, d = rp[v], rp[v + 1] - rp[v]
        lst = [int(x) for x in rl[o:o + d]]
        assert sorted(lst) == sorted(b.adj[v])
        for i in range(d - 1):
            assert b.above(lst[i], lst[i + 1]), (v, lst)
        for i in range(d):
            assert int(rk[o + i]) == len(b.N(v, col[o + i]))
        assert gam[v] == b.gamma_v(v)
        wts = [len(b.N(v, u)) * len(b.N(u, v)) for u in col[o:o + d]]
        assert sum(wts) == gam[v]
    assert g.Gamma_min == sum(1 for _ in b.tuples())


def vertex_branches(vt, n):
    """(count over 2^192, x_level, x0, x1, v) of every branch of a two-level
    vertex draw (level word, column word, threshold word)."""
    nh, TL = vt["nh"], vt["TL"]
    levels = [(TWO64, 0, 0, n)] if nh == 0 else (
        ([(TL, 0, nh, n - nh)] if TL > 0 else []) + [(TWO64 - TL, TWO64 - 1, 0, nh)])
    for cl, xl, base, m in levels:
        for c in range(m):
            cc = ic(c, m)
            t = int(vt["T"][base + c])
            if t > 0:
                yield cl * cc * t, xl, iw(c, m), 0, int(vt["self"][base + c])
            if TWO64 - t > 0:
                yield cl * cc * (TWO64 - t), xl, iw(c, m), TWO64 - 1, int(vt["alias"][base + c])


@pytest.mark.parametrize("vsplit", [oracle.ONE_LEVEL, oracle.VSPLIT, 2])
@pytest.mark.parametrize("gi", range(5))
def test_distribution_is_uniform_over_tuples(gi, vsplit):
    """Exact distribution of the oracle's draws: P(s) = tuples(s) / Gamma-check,
    P(r = w) = collision tuples / Gamma-check, and c(s) = tuples(s) / 2."""
    rp, col = tiny_graphs()[gi]
    b = Brute(rp, col)
    g = oracle.OracleGraph(rp, col, vsplit=vsplit)
    Gm = g.build_min()
    if Gm == 0:
        pytest.skip("no admissible tuple")
    rl, rk, cthr, calias, gam = g.min_tables()
    vt = g.vertex_table(3)
    rpi = [int(x) for x in rp]
    n = b.n
    probs = defaultdict(int)
    cvals = {}
    for p0, xl, x0, x1, v in vertex_branches(vt, n):
        o, d = rpi[v], b.deg[v]
        assert gam[v] > 0, "zero-weight vertex drawn"
        for j in range(d):
            cj = ic(j, d)
            keep = iw(int(cthr[o + j]), gam[v])
            sub = []
            if keep > 0:
                sub.append((cj * keep, iw(j, d), 0, j))
            if TWO64 - keep > 0:
                sub.append((cj * (TWO64 - keep), iw(j, d), TWO64 - 1, int(calias[o + j])))
            for p1, x2, x3, iu in sub:
                dvu = int(rk[o + iu])
                assert dvu > 0, "zero-weight neighbour drawn"
                u = int(g.col[o + iu])
                duv = len(b.N(u, v))
                for jw in range(dvu):
                    for jr in range(duv):
                        verts, cls = g.sample_words(oracle.MOSS4MIN, [x0, x1, x2, x3, iw(jw, dvu), iw(jr, duv),
                                                                      xl])
                        assert verts[0] == v and verts[1] == u
                        assert verts[2] in b.N(v, u) and verts[3] in b.N(u, v)
                        key = frozenset(verts[:4]) if cls else "miss"
                        probs[key] += p0 * p1 * ic(jw, dvu) * ic(jr, duv)
                        if cls:
                            cvals.setdefault(key, set()).add((cls, verts[4]))
    assert sum(probs.values()) == 1 << 448
    onto = defaultdict(int)
    miss = 0
    for v, u, w, r in b.tuples():
        if r == w:
            miss += 1
        else:
            onto[frozenset((v, u, w, r))] += 1
    for s, t in onto.items():
        ideal = Fraction(t, Gm)
        got = Fraction(probs[s], 1 << 448)
        assert abs(got - ideal) <= ideal * Fraction(1, 10 ** 12), (s, float(got), float(ideal))
    assert set(k for k in probs if k != "miss") == set(onto)
    assert abs(Fraction(probs.get("miss", 0), 1 << 448) - Fraction(miss, Gm)) <= Fraction(1, 10 ** 12)
    cis = brute_force_cis(rp, col, 4)
    for s, seen in cvals.items():
        assert len(seen) == 1, (s, seen)
        cls, c = next(iter(seen))
        assert cls == cis[s]
        if cls in (3, 5, 6):
            assert 2 * c == onto[s], (s, c, onto[s])
            if cls == 3:
                assert c == 1            # Theorem 4: 4-cycles
            if cls == 6:
                assert c == 3            # Theorem 4: 4-cliques
        else:
            assert c == 0
    # exact unbiasedness of the finalize step under this distribution
    expected = np.zeros(22)
    for s, pr in probs.items():
        if s == "miss":
            continue
        cls, c = next(iter(cvals[s]))
        sl = oracle.min_slot(cls, c)
        if sl >= 0:
            expected[sl] += pr / float(1 << 448)
    res = oracle.finalize_moss4min(np.zeros(22), expected, 0, 1, 0, Gm, 0)
    eta = np.zeros(22)
    for i in (3, 5, 6):
        eta[i] = sum(1 for s, c in cis.items() if c == i)
        assert res["eta2"][i] == pytest.approx(eta[i], rel=1e-9, abs=1e-9), i
    # with the exact counts plugged in, the reported variance of one sample is
    # sum_s 1/P(s) - n_i^2 = sum_s Gamma-check / tuples(s) - n_i^2
    res = oracle.finalize_moss4min(np.zeros(22), expected, 0, 1, 0, Gm, 0, eta=eta)
    for i in (3, 5, 6):
        ss = [s for s, c in cis.items() if c == i]
        if not ss:
            continue
        assert res["h"][i] == pytest.approx(np.mean([2.0 / onto[s] for s in ss]), rel=1e-9)
        exact = sum(Fraction(Gm, onto[s]) for s in ss) - int(eta[i]) ** 2
        assert res["var"][i] == pytest.approx(float(exact), rel=1e-9, abs=1e-9), i


def test_theorem4_counterexample_diamond():
    """A diamond whose degree-2 vertices outrank the chord is drawn 6 ways."""
    rp, col = decorated_diamond()
    b = Brute(rp, col)
    onto = sum(1 for t in b.tuples() if frozenset(t) == frozenset((0, 1, 2, 3)))
    assert onto == 6
    g = oracle.OracleGraph(rp, col)
    counts, cls, verts = g.run(oracle.MOSS4MIN, 5, 4000, record=True)
    hit = [i for i in range(len(cls)) if frozenset(verts[i, :4]) == frozenset((0, 1, 2, 3))]
    assert hit and all(cls[i] == 5 and verts[i, 4] == 3 for i in hit)
    assert counts[oracle.min_slot(5, 3)] == len(hit)
    assert counts.sum() == len(hit)


@pytest.mark.parametrize("n", [4, 5, 7, 10])
def test_complete_graph_closed_form(n):
    rp, col = synth.complete(n)
    g = oracle.OracleGraph(rp, col)
    assert g.build_min() == 6 * math.comb(n, 4) + 2 * math.comb(n, 3)
    counts, cls, verts = g.run(oracle.MOSS4MIN, 9, 3000, record=True)
    ok = cls != 0
    assert np.all(cls[ok] == 6) and np.all(verts[ok, 4] == 3)
    # a tuple lands on a clique with probability 6 C(n,4) / Gamma-check
    q = 6 * math.comb(n, 4) / g.Gamma_min
    assert abs(ok.mean() - q) < Z * math.sqrt(q * (1 - q) / 3000) + 1e-12
    assert counts[oracle.min_slot(6, 3)] == ok.sum()


def test_four_cycle_is_exact():
    rp, col = synth.cycle(4)
    g = oracle.OracleGraph(rp, col)
    assert g.build_min() == 2
    r = g.estimate_min(1000, 1000, 3)
    assert r["eta2"][3] == 1.0 and r["est"][3] == pytest.approx(1.0)
    assert r["var"][3] == pytest.approx(0.0, abs=1e-12)


def test_star_has_no_tuples():
    rp, col = synth.star(6)
    g = oracle.OracleGraph(rp, col)
    assert g.build_min() == 0
    with pytest.raises(ValueError):
        g.run(oracle.MOSS4MIN, 1, 10)
    r = g.estimate_min(100, 100, 1)
    assert r["K"] == (0, 0) and r["est"][2] == 20.0


def test_sampled_frequencies_follow_tuples():
    """Chi-square of the oracle's sampled tuples against the uniform law on the
    Gamma-check admissible tuples (the words of the real schedule)."""
    rp, col = tiny_graphs()[3]
    b = Brute(rp, col)
    g = oracle.OracleGraph(rp, col)
    Gm = g.build_min()
    allt = list(b.tuples())
    assert len(allt) == Gm
    idx = {t: i for i, t in enumerate(allt)}
    N = 200_000
    _, cls, verts = g.run(oracle.MOSS4MIN, 77, N, record=True)
    hist = np.zeros(len(allt))
    for row in verts:
        hist[idx[(int(row[0]), int(row[1]), int(row[2]), int(row[3]))]] += 1
    e = N / Gm
    chi2 = float(((hist - e) ** 2 / e).sum())
    dof = Gm - 1
    assert abs(chi2 - dof) < Z * math.sqrt(2 * dof), (chi2, dof)


@pytest.fixture(scope="module")
def g_small():
    rp, col = synth.chung_lu(120, 2.2, 7.0, 30.0, seed=5)
    b = Brute(rp, col)
    cis = brute_force_cis(rp, col, 4)
    n = np.zeros(22)
    for s, c in cis.items():
        n[c] += 1
    # S_i = sum over class-i CIS of Gamma-check / (2 c(s)), c(s) = tuples(s) / 2
    onto = defaultdict(int)
    for v, u, w, r in b.tuples():
        if r != w:
            onto[frozenset((v, u, w, r))] += 1
    g = oracle.OracleGraph(rp, col)
    Gm = g.build_min()
    S = np.zeros(22)
    for s, t in onto.items():
        if cis[s] in (3, 5, 6):
            S[cis[s]] += Gm / t
    return g, n, S


def test_variance_of_min_estimator(g_small):
    g, n, S = g_small
    R, Km = 400, 3000
    est = []
    for s in range(R):
        mm = g.run(oracle.MOSS4MIN, 10_000 + s, Km)
        est.append(oracle.finalize_moss4min(np.zeros(22), mm, 0, Km, 0, g.Gamma_min, 0)["eta2"])
    est = np.array(est)
    for i in (3, 5, 6):
        if n[i] == 0:
            continue
        V = (S[i] - n[i] ** 2) / Km            # Theorem 5 with per-CIS probabilities
        assert abs(est[:, i].mean() - n[i]) < Z * math.sqrt(V / R), (i, est[:, i].mean(), n[i])
        ratio = est[:, i].var(ddof=1) / V
        assert abs(ratio - 1) < Z * math.sqrt(2 / (R - 1) + 0.3), (i, ratio)


def test_mix_with_moss4(g_small):
    """Theorem 1 mix: nearly unbiased, and at least as accurate as the better
    of the two estimators; its reported variance tracks the sampled one."""
    g, n, S = g_small
    R, K, Km = 300, 4000, 4000
    mix, e4, em, vr = [], [], [], []
    for s in range(R):
        r = g.estimate_min(K, Km, 50_000 + s)
        mix.append(r["est"])
        e4.append(r["eta1"])
        em.append(r["eta2"])
        vr.append(r["var"])
    mix, e4, em, vr = map(np.array, (mix, e4, em, vr))
    for i in (3, 5, 6):
        if n[i] == 0:
            continue
        sd = mix[:, i].std(ddof=1)
        assert abs(mix[:, i].mean() - n[i]) < Z * sd / math.sqrt(R) + 0.02 * n[i], i
        assert sd <= 1.2 * min(e4[:, i].std(ddof=1), em[:, i].std(ddof=1)), i
        assert 0.5 < vr[:, i].mean() / sd ** 2 < 2.0, i
    # eq. (2) with the mixed classes
    for row in mix:
        assert row[2] == pytest.approx(g.Lambda3 - row[4] - 2 * row[5] - 4 * row[6])


# --------------------------------------------------------------------------
# The plug-in e_i = (K n-hat_i + K-check n-check_i) / (K + K-check) that sets
# the Theorem 1 weights of the 4-cycle, diamond and 4-clique.  At the exact
# expectations of both count vectors -- E m_i = K 2 phi_i n_i / Gamma
# (Theorem 2) and E m_{i,c} = K-check 2 c N_{i,c} / Gamma-check, N_{i,c} the
# class-i CISes with c(s) = c counted by brute force -- both estimates, the
# plug-in and the mean of 1/c equal their exact values, so the weights and
# variances equal those computed from the exact counts.  A planted slip in the
# plug-in's denominator must fail.
# --------------------------------------------------------------------------
@pytest.fixture(scope="module")
def g_small_c():
    rp, col = synth.chung_lu(120, 2.2, 7.0, 30.0, seed=5)
    b = Brute(rp, col)
    cis = brute_force_cis(rp, col, 4)
    onto = defaultdict(int)
    for v, u, w, r in b.tuples():
        if r != w:
            onto[frozenset((v, u, w, r))] += 1
    n = np.zeros(22)
    for s, c in cis.items():
        n[c] += 1
    Nc = defaultdict(int)
    for s, t in onto.items():
        assert t % 2 == 0
        Nc[(cis[s], t // 2)] += 1
    g = oracle.OracleGraph(rp, col)
    g.build_min()
    return g, n, Nc


def _check_min_plugin_at_expectation(fin, g, n, Nc, K, Km):
    from oracle.finalize import PHI4
    m = np.zeros(22)
    for i in (1, 3, 4, 5, 6):
        m[i] = K * 2.0 * PHI4[i - 1, 0] / float(g.Gamma[0]) * n[i]
    mm = np.zeros(22)
    for (cls, c), cnt in Nc.items():
        sl = oracle.min_slot(cls, c)
        if sl >= 0:
            mm[sl] += Km * 2.0 * c * cnt / float(g.Gamma_min)
    plug = fin(m, mm, K, Km, g.Gamma[0], g.Gamma_min, g.Lambda3)
    fixed = fin(m, mm, K, Km, g.Gamma[0], g.Gamma_min, g.Lambda3, eta=n)
    checked = 0
    for i in (3, 5, 6):
        if n[i] == 0:
            continue
        hbar = sum(cnt / c for (cls, c), cnt in Nc.items() if cls == i) / n[i]
        assert plug["h"][i] == pytest.approx(hbar, rel=1e-12), i
        assert plug["eta1"][i] == pytest.approx(n[i], rel=1e-12), i
        assert plug["eta2"][i] == pytest.approx(n[i], rel=1e-12), i
        assert plug["plug"][i] == pytest.approx(n[i], rel=1e-12), i
        assert plug["lam"][0, i] == pytest.approx(fixed["lam"][0, i], rel=1e-12), i
        assert plug["lam"][1, i] == pytest.approx(fixed["lam"][1, i], rel=1e-12), i
        assert plug["var"][i] == pytest.approx(fixed["var"][i], rel=1e-12), i
        checked += 1
    assert checked >= 2


@pytest.mark.parametrize("K,Km", [(4000, 4000), (1000, 9000), (9000, 700)])
def test_min_plugin_exact_at_expected_counts(g_small_c, K, Km):
    g, n, Nc = g_small_c
    _check_min_plugin_at_expectation(oracle.finalize_moss4min, g, n, Nc, K, Km)


def test_min_plugin_pin_catches_a_planted_slip(g_small_c):
    import inspect
    g, n, Nc = g_small_c
    src = inspect.getsource(oracle.finalize)
    good = "e = (K * e4[i] + Kmin * em[i]) / (K + Kmin)"
    assert src.count(good) == 1
    ns: dict = {}
    exec(compile(src.replace(good, "e = (K * e4[i] + Kmin * em[i]) / (2 * K)"), "planted", "exec"), ns)
    with pytest.raises(AssertionError):
        _check_min_plugin_at_expectation(ns["finalize_moss4min"], g, n, Nc, 1000, 9000)
