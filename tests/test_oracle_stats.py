"""Statistical pins of the oracle's estimators against exact ESU counts (CPU).

* Unbiasedness (Theorems 3, 7, 9, 10): the mean over R independent seeds lies
  within z sigma / sqrt(R) of the exact count, sigma^2 being the paper's
  variance evaluated at the exact counts.
* Variances: the empirical variance over R = 1000 seeds, divided by the
  closed form at the exact counts, lies in the band
  1 +- z sqrt(2/(R-1) + kappa/R), kappa the excess kurtosis of the scaled
  binomial count (the chi^2_{R-1}/(R-1) band widened for non-normality).
z = 4.5 keeps the family-wise false-alarm rate far below 1% over all classes.
"""
from __future__ import annotations

import json
import math
import os

import numpy as np
import pytest

import oracle
import synth
from oracle.finalize import PHI4, PHI5

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "esu_counts.json")))
Z = 4.5


def var_moss4(eta, K, G):
    v = np.zeros(7)
    p = np.zeros(7)
    for i in (1, 3, 4, 5, 6):
        p[i] = 2 * PHI4[i - 1, 0] / G
        v[i] = eta[i] / K * (1 / p[i] - eta[i])
    v[2] = (eta[4] / p[4] + 4 * eta[5] / p[5] + 16 * eta[6] / p[6] - (eta[4] + 2 * eta[5] + 4 * eta[6]) ** 2) / K
    return v, p


def kurt(q, K):
    q = min(max(q, 1e-300), 1 - 1e-16)
    return (1 - 6 * q * (1 - q)) / (K * q * (1 - q))


@pytest.fixture(scope="module")
def g200():
    rp, col = synth.chung_lu(200, 2.3, 6.0, 30.0, seed=7)
    g = oracle.OracleGraph(rp, col)
    assert str(g.Gamma[0]) == GOLD["cl_n200"]["Gamma"][0]
    return g


def test_moss4_unbiased_on_n2k_workload():
    rp, col = synth.workload("cl_n2k")
    g = oracle.OracleGraph(rp, col)
    eta = np.array(GOLD["cl_n2k"]["esu4"], dtype=np.float64)
    R, K = 30, 100_000
    est = np.array([g.estimate(4, K, seed=1000 + s)["est"] for s in range(R)])
    v, _ = var_moss4(eta, K, float(g.Gamma[0]))
    for i in range(1, 7):
        assert abs(est[:, i].mean() - eta[i]) < Z * math.sqrt(v[i] / R), (i, est[:, i].mean(), eta[i])


def test_moss4_variance_matches_theorem3(g200):
    eta = np.array(GOLD["cl_n200"]["esu4"], dtype=np.float64)
    R, K = 1000, 2000
    est = np.array([g200.estimate(4, K, seed=s)["est"] for s in range(R)])
    G = float(g200.Gamma[0])
    v, p = var_moss4(eta, K, G)
    for i in range(1, 7):
        assert abs(est[:, i].mean() - eta[i]) < Z * math.sqrt(v[i] / R), i
        q = p[i] * eta[i] if i != 2 else None
        if i != 2 and K * q < 30:
            continue
        k = kurt(q, K) if i != 2 else 0.05
        ratio = est[:, i].var(ddof=1) / v[i]
        assert abs(ratio - 1) < Z * math.sqrt(2 / (R - 1) + k / R), (i, ratio)


def test_moss5_fixed_lambda_matches_theorem10(g200):
    """With lambda computed from the exact counts (a constant), the mix
    estimator is exactly unbiased and its variance is Theorem 10's."""
    eta = np.array(GOLD["cl_n200"]["esu5"], dtype=np.float64)
    R, B = 1000, 4000
    runs = [g200.estimate(5, B, seed=s, eta=eta) for s in range(R)]
    est = np.array([r["est"] for r in runs])
    ref = runs[0]
    K1, K2 = ref["K"]
    p = ref["p"]
    for i in range(1, 22):
        v = ref["var"][i]               # closed form at the exact counts
        assert abs(est[:, i].mean() - eta[i]) < Z * math.sqrt(v / R) + 1e-9, (i, est[:, i].mean(), eta[i])
        if i == 2:
            ratio = est[:, i].var(ddof=1) / v
            assert abs(ratio - 1) < Z * math.sqrt(2 / (R - 1) + 0.05 / R), ratio
            continue
        q = [p[l, i] * eta[i] for l in range(2)]
        hits = [K1 * q[0], K2 * q[1]]
        if max(hits) < 30:
            continue
        k = max(kurt(q[l], (K1, K2)[l]) for l in range(2) if q[l] > 0)
        ratio = est[:, i].var(ddof=1) / v
        assert abs(ratio - 1) < Z * math.sqrt(2 / (R - 1) + k / R), (i, ratio)
    # Cov(eta_i, eta_j) of Theorem 10 on the most correlated pairs; the
    # sample covariance has variance ~ (V_i V_j + C_ij^2) / R
    cov = ref["cov"]
    cand = [i for i in range(1, 22) if i != 2 and ref["var"][i] > 0]
    pairs = sorted(((abs(cov[i, j]) / math.sqrt(ref["var"][i] * ref["var"][j]), i, j)
                    for i in cand for j in cand if i < j), reverse=True)[:3]
    for corr, i, j in pairs:
        assert corr > 0.1
        emp = np.cov(est[:, i], est[:, j])[0, 1]
        se = math.sqrt((ref["var"][i] * ref["var"][j] + cov[i, j] ** 2) / R)
        assert abs(emp - cov[i, j]) < Z * se, (i, j, emp, cov[i, j])


def test_moss5_plugin_lambda_is_nearly_unbiased(g200):
    """With the plug-in lambda the mix is no longer exactly unbiased
    (Theorem 10 assumes fixed weights); its bias must stay small."""
    eta = np.array(GOLD["cl_n200"]["esu5"], dtype=np.float64)
    R, B = 400, 8000
    runs = [g200.estimate(5, B, seed=5000 + s) for s in range(R)]
    est = np.array([r["est"] for r in runs])
    exact = g200.estimate(5, B, seed=0, eta=eta)
    for i in range(1, 22):
        if eta[i] == 0:
            assert np.all(est[:, i] == 0) or i == 2
            continue
        sd = math.sqrt(exact["var"][i])
        assert abs(est[:, i].mean() - eta[i]) < 6 * sd / math.sqrt(R) + 0.02 * eta[i], i


def test_sampled_classes_stay_in_omega(g200):
    m1 = g200.run(oracle.T5, 3, 50_000)
    m2 = g200.run(oracle.PATH5, 3, 50_000)
    for i in range(1, 22):
        if PHI5[i - 1, 0] == 0:
            assert m1[i] == 0
        if PHI5[i - 1, 1] == 0:
            assert m2[i] == 0
    m0 = g200.run(oracle.MOSS4, 3, 50_000)
    assert m0[2] == 0


def test_covariance_matrix_is_consistent(g200):
    """The class-2 entries of the covariance matrix follow from the identities:
    Var(n_2) of Theorem 3 equals Var(n_4 + 2 n_5 + 4 n_6) built from the
    pairwise covariances, and for k = 5 Var(eta_2) equals the quadratic form
    of the phi^(3) weights; the matrix is symmetric positive semi-definite on
    the sampled classes; concentrations sum to 1."""
    r4 = g200.estimate(4, 200_000, seed=3)
    c = np.zeros(22)
    c[4], c[5], c[6] = 1.0, 2.0, 4.0
    assert abs(c @ r4["cov"] @ c - r4["var"][2]) <= 1e-9 * abs(r4["var"][2])
    assert np.allclose(r4["cov"], r4["cov"].T)
    assert abs(r4["conc"][1:7].sum() - 1.0) < 1e-12
    r5 = g200.estimate(5, 200_000, seed=3)
    phi = np.zeros(22)
    for i in range(1, 22):
        if i != 2:
            phi[i] = PHI5[i - 1, 2]
    assert abs(phi @ r5["cov"] @ phi - r5["var"][2]) <= 1e-9 * abs(r5["var"][2])
    sub = [i for i in range(1, 22) if i != 2]
    ev = np.linalg.eigvalsh(r5["cov"][np.ix_(sub, sub)])
    assert ev.min() > -1e-9 * ev.max()
    assert abs(r5["conc"][1:22].sum() - 1.0) < 1e-12


def test_covariance_matches_sampling(g200):
    """Off-diagonal covariances of the MOSS-4 estimates against the sample
    covariance over 1,000 seeds at the exact counts (proof of Theorem 3)."""
    eta = np.array(GOLD["cl_n200"]["esu4"], dtype=np.float64)
    R, K = 1000, 2000
    est = np.array([g200.estimate(4, K, seed=s)["est"] for s in range(R)])
    ref = g200.estimate(4, K, seed=0, eta=eta)["cov"]
    for i, j in ((1, 3), (1, 4), (3, 4), (1, 2), (2, 4)):
        emp = np.cov(est[:, i], est[:, j])[0, 1]
        se = math.sqrt((ref[i, i] * ref[j, j] + ref[i, j] ** 2) / R)
        assert abs(emp - ref[i, j]) < Z * se, (i, j, emp, ref[i, j])


# --------------------------------------------------------------------------
# The pooled plug-in eta~ = (m1 + m2) / (K1 p1 + K2 p2) that sets lambda for
# the classes of Omega_1 and Omega_2 (mix estimator, Sec. 5.1.3; Theorem 10).
# Two properties fix it independently of its formula:
#  (a) it is linear in the counts and equals eta at their expectations
#      E m^(l)_i = K_l p^(l)_i eta_i (Theorems 6, 8), so it is exactly unbiased
#      and, fed those expectations, lambda equals the fixed-lambda value of
#      Theorem 10 computed from the exact counts;
#  (b) it is the maximum of the likelihood of the common eta_i given both
#      sub-methods' hit counts, each a rare-event (Poisson) count of mean
#      K_l p^(l)_i eta_i.
# A planted slip in its denominator must fail (a).
# --------------------------------------------------------------------------
def _mixed_classes():
    return [i for i in range(1, 22) if PHI5[i - 1, 0] > 0 and PHI5[i - 1, 1] > 0]


def _expected_counts(g, eta, K1, K2):
    m = np.zeros((2, 22))
    for l, K in ((0, K1), (1, K2)):
        for i in range(1, 22):
            if PHI5[i - 1, l] > 0:
                m[l, i] = K * 2.0 * PHI5[i - 1, l] / float(g.Gamma[1 + l]) * eta[i]
    return m


def _check_plugin_at_expectation(fin, g, eta, K1, K2):
    m = _expected_counts(g, eta, K1, K2)
    plug = fin(m[0], m[1], K1, K2, g.Gamma[1], g.Gamma[2], g.Lambda4)
    fixed = fin(m[0], m[1], K1, K2, g.Gamma[1], g.Gamma[2], g.Lambda4, eta=eta)
    for i in _mixed_classes():
        if eta[i] == 0:
            continue
        # the single-source estimates agree (both eta_i) and the pooled value equals them
        assert plug["eta1"][i] == pytest.approx(eta[i], rel=1e-12)
        assert plug["eta2"][i] == pytest.approx(eta[i], rel=1e-12)
        assert plug["plug"][i] == pytest.approx(eta[i], rel=1e-12), i
        assert plug["lam"][0, i] == pytest.approx(fixed["lam"][0, i], rel=1e-12), i
        assert plug["lam"][1, i] == pytest.approx(fixed["lam"][1, i], rel=1e-12), i
        assert plug["var"][i] == pytest.approx(fixed["var"][i], rel=1e-12), i


@pytest.mark.parametrize("K1,K2", [(4000, 4000), (1000, 9000), (12345, 321)])
def test_pooled_plugin_exact_at_expected_counts(g200, K1, K2):
    eta = np.array(GOLD["cl_n200"]["esu5"], dtype=np.float64)
    assert sum(eta[i] > 0 for i in _mixed_classes()) >= 5
    _check_plugin_at_expectation(oracle.finalize_moss5, g200, eta, K1, K2)


def test_pooled_plugin_is_the_joint_likelihood_maximum(g200):
    from scipy.optimize import minimize_scalar
    K1, K2 = 30_000, 20_000
    m1 = g200.run(oracle.T5, 17, K1).astype(np.float64)
    m2 = g200.run(oracle.PATH5, 17, K2).astype(np.float64)
    r = oracle.finalize_moss5(m1, m2, K1, K2, g200.Gamma[1], g200.Gamma[2], g200.Lambda4)
    checked = 0
    for i in _mixed_classes():
        if m1[i] + m2[i] == 0:
            assert r["plug"][i] == 0.0
            continue
        rate = np.array([K1 * r["p"][0, i], K2 * r["p"][1, i]])
        cnt = np.array([m1[i], m2[i]])

        def nll(x):
            return float(np.sum(rate * x - cnt * np.log(rate * x)))
        hi = 10.0 * (cnt.sum() + 1) / rate.min()
        opt = minimize_scalar(nll, bounds=(1e-12 * hi, hi), method="bounded",
                              options={"xatol": 1e-10 * hi, "maxiter": 500})
        assert opt.x == pytest.approx(r["plug"][i], rel=1e-6), i
        checked += 1
    assert checked >= 5


def test_pooled_plugin_pin_catches_a_planted_slip(g200):
    """The pin above fails on a copy of the oracle's finalize whose pooled
    denominator is (K1 + K2) p^(1) instead of K1 p^(1) + K2 p^(2)."""
    import inspect
    src = inspect.getsource(oracle.finalize)
    good = "e = (m1[i] + m2[i]) / (K1 * p[0, i] + K2 * p[1, i])"
    assert src.count(good) == 1
    ns: dict = {}
    exec(compile(src.replace(good, "e = (m1[i] + m2[i]) / ((K1 + K2) * p[0, i])"), "planted", "exec"), ns)
    eta = np.array(GOLD["cl_n200"]["esu5"], dtype=np.float64)
    with pytest.raises(AssertionError):
        _check_plugin_at_expectation(ns["finalize_moss5"], g200, eta, 4000, 4000)
