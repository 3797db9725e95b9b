"""The budget rule of the request server (host arithmetic, no GPU): the
samples at which the relative standard error of Theorem 3 (and 7, 9),
sqrt((1/(p_i n_i) - 1) / K), reaches the target for every class with at least
10 pilot hits (p_i n_i estimated by the pilot hit fraction)."""
from __future__ import annotations

import math

import numpy as np

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
