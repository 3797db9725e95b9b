"""The budget rule of the request server (host arithmetic, no GPU): the
samples at which the relative standard error of Theorem 3 (and 7, 9),
sqrt((1/(p_i n_i) - 1) / K), reaches the target for every class with at least
10 pilot hits (p_i n_i estimated by the pilot hit fraction)."""
from __future__ import annotations

import math

import numpy as np

import pytest

import paper_1509_08089_gb300 as moss


def rule(k, K, hits, eps, lo, hi):
    need = 0.0
    for l in range(1 if k == 4 else 2):
        if K[l] == 0:
            continue
        for i in range(1, 22):
            m = int(hits[l][i])
            if m >= 10:
                f = m / K[l]
                need = max(need, (1 / f - 1) / eps ** 2 * (2 if k == 5 else 1))
    return int(min(max(math.ceil(need), lo), hi))


def test_budget_rule_matches_theorem3():
    rng = np.random.default_rng(4)
    for _ in range(200):
        k = int(rng.choice([4, 5]))
        K = [int(rng.integers(1_000, 100_000)), int(rng.integers(1_000, 100_000)) if k == 5 else 0]
        hits = np.zeros((2, 22), dtype=np.uint64)
        for l in range(2 if k == 5 else 1):
            hits[l, 1:] = rng.multinomial(K[l], rng.dirichlet(np.ones(21) * 0.3))
        eps = float(rng.uniform(0.01, 0.05))
        got = moss.moss_budget_for_target(k, K, hits, eps, 10_000, 10_000_000)
        assert got == rule(k, K, hits, eps, 10_000, 10_000_000)


def test_budget_reaches_target_when_unclamped():
    # one class at hit fraction f: K (1/f - 1)^-1 eps^2 = 1 means relative SE = eps
    K = [100_000, 0]
    hits = np.zeros((2, 22), dtype=np.uint64)
    hits[0][1] = 1_000          # f = 0.01
    hits[0][3] = 99_000
    b = moss.moss_budget_for_target(4, K, hits, 0.02, 1, 10**12)
    f = 0.01
    assert abs(math.sqrt((1 / f - 1) / b) - 0.02) < 1e-6


def test_min_budget_reaches_target_by_the_oracle_variance():
    """The MOSS-4 + MOSS-4Min budget rule against the oracle's variance of
    the mixed estimate (Theorems 1, 3 and 5): with pilot counts at their
    expectations, the budget B it returns gives, at K = K-check = B / 2 and
    the exact counts plugged in, a relative standard error of exactly eps for
    the class that sets B and at most eps for the others."""
    from collections import defaultdict

    import oracle
    import synth
    from helpers import brute_force_cis
    from test_oracle_min import Brute
    rp, col = synth.chung_lu(120, 2.2, 7.0, 30.0, seed=5)
    b = Brute(rp, col)
    cis = brute_force_cis(rp, col, 4)
    n = np.zeros(22)
    for s, c in cis.items():
        n[c] += 1
    onto = defaultdict(int)
    for v, u, w, r in b.tuples():
        if r != w:
            onto[frozenset((v, u, w, r))] += 1
    og = oracle.OracleGraph(rp, col)
    Gm = og.build_min()
    G = og.Gamma[0]
    Kp = 10 ** 9                   # pilot size at which rounding the expectations is negligible
    hits = np.zeros((2, 22))
    for i in (1, 3, 4, 5, 6):
        hits[0][i] = round(Kp * 2 * oracle.PHI4[i - 1, 0] * n[i] / G)
    for s, t in onto.items():
        sl = oracle.min_slot(cis[s], t // 2)
        if sl >= 0:
            hits[1][sl] += Kp * 2 * (t // 2) / Gm
    hits[1] = np.round(hits[1])
    eps = 0.02
    B = moss.moss_budget_for_target_min([Kp, Kp], hits.astype(np.uint64), eps, 1, 10 ** 15)
    K, Km = B // 2, B - B // 2
    mm = np.zeros(22)
    for s, t in onto.items():
        sl = oracle.min_slot(cis[s], t // 2)
        if sl >= 0:
            mm[sl] += Km * 2 * (t // 2) / Gm
    m = np.zeros(22)
    for i in (1, 3, 4, 5, 6):
        m[i] = K * 2 * oracle.PHI4[i - 1, 0] * n[i] / G
    r = oracle.finalize_moss4min(m, mm, K, Km, G, Gm, og.Lambda3, eta=n)
    rse = [np.sqrt(r["var"][i]) / n[i] for i in (1, 3, 4, 5, 6) if n[i] > 0]
    assert max(rse) == pytest.approx(eps, rel=2e-3)
    assert all(x <= eps * (1 + 2e-3) for x in rse)


def test_min_budget_without_enough_hits_is_the_minimum():
    hits = np.zeros((2, 22), dtype=np.uint64)
    hits[0][1] = 9
    hits[1][0] = 9
    assert moss.moss_budget_for_target_min([1000, 1000], hits, 0.01, 12_345, 10 ** 7) == 12_345
    hits[0][1] = 500          # f = 0.5: 1/f - 1 = 1, B = 2 / eps^2
    assert moss.moss_budget_for_target_min([1000, 1000], hits, 0.01, 1, 10 ** 9) == 20_000
    assert moss.moss_budget_for_target_min([1000, 1000], hits, 0.01, 1, 15_000) == 15_000
