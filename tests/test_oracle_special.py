"""Closed-form special cases of the estimators (CPU, oracle only).

* Cycle C_n (n >= 6): every MOSS-4 sample is a 3-path, so n_1 = n exactly
  with variance 0 (Theorem 3 with p_1 = 2/Gamma, Gamma = 2n); every Path-5
  sample is a 5-path, eta_1 = n exactly; Gamma^(1) = 0 so T-5 is idle.
* Star K_{1,m}: Gamma = Gamma^(1) = Gamma^(2) = 0, so n_2 = Lambda_3 = C(m,3)
  and eta_2 = Lambda_4 = C(m,4) exactly (eq. 2, Sec. 5.1.3).
* Complete K_n: MOSS-4 hits M_6 with probability (n-3)/(n-2) per sample, the
  rest are triangles (r = w); T-5 hits M_21 with probability (n-4)/(n-2).
"""
from __future__ import annotations

import math

import numpy as np
import pytest

import oracle
import synth


@pytest.mark.parametrize("n", [6, 10, 31])
def test_cycle_is_exact(n):
    g = oracle.OracleGraph(*synth.cycle(n))
    r4 = g.estimate(4, 5000, seed=3)
    assert r4["est"][1] == pytest.approx(n, rel=0, abs=1e-9)
    assert r4["var"][1] == pytest.approx(0.0, abs=1e-9)
    assert all(r4["est"][i] == 0 for i in (2, 3, 4, 5, 6))
    r5 = g.estimate(5, 5000, seed=3)
    assert r5["K"][0] == 0                       # Gamma^(1) = 0: no fork exists
    assert r5["est"][1] == pytest.approx(n, abs=1e-9)
    assert r5["var"][1] == pytest.approx(0.0, abs=1e-9)
    assert all(r5["est"][i] == 0 for i in range(2, 22))


@pytest.mark.parametrize("m", [3, 4, 9])
def test_star_is_exact(m):
    g = oracle.OracleGraph(*synth.star(m))
    r4 = g.estimate(4, 1000, seed=1)
    assert r4["K"][0] == 0
    assert r4["est"][2] == math.comb(m, 3)
    assert r4["var"][2] == 0
    r5 = g.estimate(5, 1000, seed=1)
    assert r5["est"][2] == math.comb(m, 4)
    assert r5["var"][2] == 0


@pytest.mark.parametrize("n", [6, 8])
def test_complete_graph_hit_rates(n):
    g = oracle.OracleGraph(*synth.complete(n))
    K = 200_000
    m = g.run(oracle.MOSS4, 9, K)
    p = (n - 3) / (n - 2)
    assert abs(m[6] / K - p) < 5 * math.sqrt(p * (1 - p) / K)
    assert m[6] + m[0] == K
    r = g.estimate(4, K, seed=9)
    sd = math.sqrt(r["var"][6])
    assert abs(r["est"][6] - math.comb(n, 4)) < 5 * sd
    # K_n has no 3-star CIS: n_2 = Lambda_3 - 4 n_6 (eq. 2) must be ~0
    assert abs(r["est"][2]) < 5 * math.sqrt(r["var"][2]) + 1e-9
    # and no 4-star CIS: eta_2 = Lambda_4 - 5 eta_21 (Table 2 row 21)
    r5 = g.estimate(5, K, seed=9)
    assert abs(r5["est"][21] - math.comb(n, 5)) < 5 * math.sqrt(r5["var"][21])
    assert abs(r5["est"][2]) < 5 * math.sqrt(r5["var"][2]) + 1e-9
    m5 = g.run(oracle.T5, 9, K)
    p5 = (n - 4) / (n - 2)
    assert abs(m5[21] / K - p5) < 5 * math.sqrt(p5 * (1 - p5) / K)
    m6 = g.run(oracle.PATH5, 9, K)
    # Path-5 on K_n: r, t are uniform in N_u-{v}, N_w-{v}; collisions r=w,
    # t=u, t=r each have probability 1/(n-2) and are disjoint except t=r=...
    assert m6[21] + m6[0] == K


def test_triangle_estimator_unbiased():
    rp, col = synth.chung_lu(400, 2.4, 8.0, 60.0, seed=2)
    g = oracle.OracleGraph(rp, col)
    adj = [set(col[int(rp[v]):int(rp[v + 1])].tolist()) for v in range(400)]
    T = sum(1 for a in range(400) for b in adj[a] if b > a for c in adj[b] if c > b and c in adj[a])
    R, K = 200, 5000
    ests = [g.estimate(4, K, seed=s)["triangles"] for s in range(R)]
    G = g.Gamma[0]
    sd = math.sqrt(T / K * (G / 6 - T))
    assert abs(np.mean(ests) - T) < 4.5 * sd / math.sqrt(R)
