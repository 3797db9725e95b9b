"""Estimators and variances (FP64) -- part of the test oracle.

Everything is written as the paper states it, in a fixed evaluation order:

* MOSS-4 (Sec. 4.1.2, Theorem 2, Theorem 3): p_i = 2 phi_i^(1) / Gamma,
  n_i = m_i / (K p_i) for i in {1,3,4,5,6}; n_2 = Lambda_3 - n_4 - 2 n_5 - 4 n_6
  (eq. 2); Var(n_i) = n_i/K (1/p_i - n_i); Var(n_2) per Theorem 3.
  Also the triangle count implied by the collisions r = w: each triangle is
  produced by 6 ordered (v, u, w) draws of probability 1/Gamma each (the
  argument of the proof of Theorem 2), so T = m_0 Gamma / (6 K).
* MOSS-4Min (Sec. 4.2, Algorithm 2, Theorem 5) with one correction: a CIS
  s of class 3, 5 or 6 is drawn with probability 2 c(s) / Gamma-check, where
  c(s) counts the 3-paths p0-p1-p2-p3 of s with p0 > p2 and p3 > p1 in the
  total order (each drawn from both of its orientations).  c is 1 for every
  4-cycle and 3 for every 4-clique, as Theorem 4 states, but 1, 2 or 3 for a
  diamond, so counts are kept per (class, c) slot and each hit has the
  Horvitz-Thompson weight Gamma-check / (2 c).  Theorem 5 becomes
  Var = (sum_s 1/P(s) - n_i^2) / K-check; the mix with MOSS-4 follows
  Theorem 1.
* MOSS-5 (Sec. 5.1, Theorems 6-10): eta^(l)_i = m^(l)_i / (K_l p^(l)_i),
  p^(l)_i = 2 phi^(l)_i / Gamma^(l); the mix estimator (eq. mixestimator)
  with lambda from the two variances; eta_2 = Lambda_4 - sum phi^(3)_i eta_i
  over Omega_3* and its variance from Theorem 10.

The variances contain the unknown eta_i; the plug-in value is the estimate
itself for a single-source class and the pooled value
(m1 + m2) / (K1 p1 + K2 p2) for a class of Omega_1 and Omega_2, so that a
class seen by only one sub-method keeps a positive weight on it.  Passing
``eta=...`` replaces the plug-in by given values (e.g. the exact counts, with
which lambda is a constant and Theorem 10 holds exactly).
"""
from __future__ import annotations

import numpy as np

# Sec. 4.1.2: phi^(1) (copies of M_1^(4)) and phi^(2) (copies of M_2^(4)) of M_1..M_6.
PHI4 = np.array([[1, 0], [0, 1], [4, 0], [2, 1], [6, 2], [12, 4]], dtype=np.float64)
# Table 2: phi^(1) (forks), phi^(2) (5-paths), phi^(3) (4-stars) of M_1^(5)..M_21^(5).
PHI5 = np.array([
    [0, 1, 0], [0, 0, 1], [1, 0, 0], [1, 2, 0], [2, 2, 0], [0, 5, 0], [2, 1, 0],
    [2, 0, 1], [4, 4, 0], [4, 7, 0], [5, 2, 1], [4, 4, 1], [6, 6, 0], [10, 10, 1],
    [9, 6, 1], [12, 6, 2], [10, 14, 0], [20, 24, 1], [20, 18, 2], [36, 36, 3], [60, 60, 5]],
    dtype=np.float64)


def finalize_moss4(m, K: int, Gamma: int, Lambda3: int, eta=None) -> dict:
    """m: counts[22] with m[0] = collisions (triangles), m[i] class i."""
    m = np.asarray(m, dtype=np.float64)
    G = float(Gamma)
    est = np.zeros(7)
    var = np.zeros(7)
    p = np.zeros(7)
    sampled = (1, 3, 4, 5, 6)
    tri = 0.0
    tri_var = 0.0
    if K > 0 and G > 0:
        for i in sampled:
            p[i] = 2.0 * PHI4[i - 1, 0] / G                 # Theorem 2
            est[i] = m[i] / (K * p[i])                       # Sec. 4.1.2
        plug = est if eta is None else np.asarray(eta, dtype=np.float64)
        for i in sampled:
            var[i] = plug[i] / K * (1.0 / p[i] - plug[i])   # Theorem 3
        var[2] = (plug[4] / p[4] + 4.0 * plug[5] / p[5] + 16.0 * plug[6] / p[6]
                  - (plug[4] + 2.0 * plug[5] + 4.0 * plug[6]) ** 2) / K
        tri = m[0] * G / (6.0 * K)
        tri_var = tri / K * (G / 6.0 - tri)
    est[2] = float(Lambda3) - est[4] - 2.0 * est[5] - 4.0 * est[6]   # eq. (2)
    # covariance matrix: Cov(n_i, n_j) = -n_i n_j / K for sampled i != j
    # (proof of Theorem 3); n_2 = Lambda_3 - n_4 - 2 n_5 - 4 n_6 is linear in them
    cov = np.zeros((22, 22))
    if K > 0 and G > 0:
        plug = est if eta is None else np.asarray(eta, dtype=np.float64)
        for i in sampled:
            for j in sampled:
                cov[i, j] = var[i] if i == j else -plug[i] * plug[j] / K
        c = {4: 1.0, 5: 2.0, 6: 4.0}
        for j in range(1, 7):
            if j != 2:
                cov[2, j] = cov[j, 2] = -sum(c[i] * cov[i, j] for i in (4, 5, 6))
        cov[2, 2] = var[2]
    return {"k": 4, "K": (K, 0), "est": est, "var": var, "p": p,
            "triangles": tri, "triangles_var": tri_var, "cov": cov, "conc": concentrations(est, 6)}


def min_slot(cls: int, c: int) -> int:
    """Count slot of a MOSS-4Min hit of class cls with c(s) = c: 4-cycles
    use slots 0-3 (c = 1..4), diamonds 4-9 (c = 1..6), 4-cliques 10-21
    (c = 1..12); -1 for anything not counted."""
    if cls == 3 and 1 <= c <= 4:
        return c - 1
    if cls == 5 and 1 <= c <= 6:
        return 4 + c - 1
    if cls == 6 and 1 <= c <= 12:
        return 10 + c - 1
    return -1


MIN_CLASSES = {3: (0, 4), 5: (4, 6), 6: (10, 12)}    # class -> (first slot, slots)
# 1/c of every CIS of the class as Theorem 4 states it (4-cycles c = 1, diamonds
# c = 1, 4-cliques c = 3): the plug-in mean of 1/c for a class MOSS-4Min did not hit
THM4_INV_C = {3: 1.0, 5: 1.0, 6: 1.0 / 3.0}


def finalize_moss4min(m, mm, K: int, Kmin: int, Gamma: int, Gamma_min: int, Lambda3: int, eta=None) -> dict:
    """m: MOSS-4 counts[22]; mm: MOSS-4Min slot counts[22] (:func:`min_slot`).

    MOSS-4Min estimate of class i in {3, 5, 6} (Algorithm 2 with the weight
    Gamma-check / (2 c)): n-check_i = Gamma-check / (2 K-check) sum_c m_{i,c} / c.
    Its variance (Theorem 5 with per-CIS probabilities) is
    (S_i - n_i^2) / K-check with S_i = sum_s 1/P(s) = n_i Gamma-check h_i / 2,
    h_i the mean of 1/c(s) over the class, estimated by
    sum_c m_{i,c}/c^2 / sum_c m_{i,c}/c (THM4_INV_C when the class has no hit).
    n_i in both variances is the plug-in e_i = (K n-hat_i + K-check n-check_i)
    / (K + K-check) (or eta).  The two estimates of a class are mixed with
    weights proportional to the inverse variances (Theorem 1); classes 1 and 4
    come from MOSS-4 alone and n_2 from eq. (2)."""
    m = np.asarray(m, dtype=np.float64)
    mm = np.asarray(mm, dtype=np.float64)
    G, Gm = float(Gamma), float(Gamma_min)
    avail = (K > 0 and G > 0, Kmin > 0 and Gm > 0)
    sampled = (1, 3, 4, 5, 6)
    p = np.zeros(22)
    e4 = np.zeros(22)                     # n-hat (MOSS-4)
    em = np.zeros(22)                     # n-check (MOSS-4Min)
    h = np.zeros(22)
    if avail[0]:
        for i in sampled:
            p[i] = 2.0 * PHI4[i - 1, 0] / G                 # Theorem 2
            e4[i] = m[i] / (K * p[i])
    if avail[1]:
        for i, (s0, ns) in MIN_CLASSES.items():
            a = 0.0
            b = 0.0
            for c in range(1, ns + 1):
                a += mm[s0 + c - 1] / c
                b += mm[s0 + c - 1] / (c * c)
            em[i] = Gm / (2.0 * Kmin) * a
            h[i] = b / a if a > 0 else THM4_INV_C[i]
    est = np.zeros(22)
    var = np.zeros(22)
    lam = np.zeros((2, 22))
    plug = np.zeros(22)
    for i in sampled:
        src = [l for l in range(2) if avail[l] and (l == 0 or i in MIN_CLASSES)]
        if not src:
            continue
        if len(src) == 1:
            l = src[0]
            e = (e4[i] if l == 0 else em[i]) if eta is None else float(eta[i])
            plug[i] = e
            if l == 0:
                var[i] = e / K * (1.0 / p[i] - e)                    # Theorem 3
                est[i] = e4[i]
            else:
                var[i] = (e * Gm * h[i] / 2.0 - e * e) / Kmin        # Theorem 5, per-CIS P(s)
                est[i] = em[i]
            lam[l, i] = 1.0
            continue
        e = (K * e4[i] + Kmin * em[i]) / (K + Kmin) if eta is None else float(eta[i])
        plug[i] = e
        V1 = max(e / K * (1.0 / p[i] - e), 0.0)
        V2 = max((e * Gm * h[i] / 2.0 - e * e) / Kmin, 0.0)
        if V1 + V2 > 0.0:
            lam[0, i] = V2 / (V1 + V2)
            lam[1, i] = V1 / (V1 + V2)
            var[i] = V1 * V2 / (V1 + V2)                             # Theorem 1
        else:
            lam[0, i] = lam[1, i] = 0.5
            var[i] = 0.0
        est[i] = lam[0, i] * e4[i] + lam[1, i] * em[i]
    # a sample lands in one class: Cov = -sum_l a^(l)_i a^(l)_j n_i n_j / K_l
    cov = np.zeros((22, 22))
    Ks = (K, Kmin)
    for l in range(2):
        if avail[l]:
            a = lam[l] * plug
            cov -= np.outer(a, a) / Ks[l]
    np.fill_diagonal(cov, 0.0)
    for i in range(22):
        cov[i, i] = var[i]
    coef = {4: 1.0, 5: 2.0, 6: 4.0}
    est[2] = float(Lambda3) - est[4] - 2.0 * est[5] - 4.0 * est[6]   # eq. (2)
    v2 = 0.0
    for i in coef:
        for j in coef:
            v2 += coef[i] * coef[j] * cov[i, j]
    for j in range(1, 7):
        if j != 2:
            c2 = 0.0
            for i in coef:
                c2 -= coef[i] * cov[i, j]
            cov[2, j] = cov[j, 2] = c2
    var[2] = v2 if avail[0] or avail[1] else 0.0
    cov[2, 2] = var[2]
    tri = 0.0
    tri_var = 0.0
    if avail[0]:
        tri = m[0] * G / (6.0 * K)
        tri_var = tri / K * (G / 6.0 - tri)
    return {"k": 4, "K": (K if avail[0] else 0, Kmin if avail[1] else 0), "est": est, "var": var, "lam": lam,
            "eta1": e4, "eta2": em, "h": h, "p": p, "plug": plug, "cov": cov, "triangles": tri,
            "triangles_var": tri_var, "conc": concentrations(est, 6)}


def concentrations(est, n_classes: int) -> np.ndarray:
    """omega_i = eta_i / sum_j eta_j over the classes (Sec. 6.3)."""
    out = np.zeros(22)
    tot = 0.0
    for i in range(1, n_classes + 1):
        tot += est[i]
    if tot != 0.0:
        for i in range(1, n_classes + 1):
            out[i] = est[i] / tot
    return out


def finalize_moss5(m1, m2, K1: int, K2: int, Gamma1: int, Gamma2: int, Lambda4: int, eta=None) -> dict:
    """m1, m2: counts[22] of T-5 and Path-5 ([0] = collisions)."""
    m1 = np.asarray(m1, dtype=np.float64)
    m2 = np.asarray(m2, dtype=np.float64)
    G = (float(Gamma1), float(Gamma2))
    K = (K1, K2)
    mm = (m1, m2)
    avail = (K1 > 0 and G[0] > 0, K2 > 0 and G[1] > 0)
    p = np.zeros((2, 22))
    eh = np.zeros((2, 22))
    for l in range(2):
        if not avail[l]:
            continue
        for i in range(1, 22):
            if PHI5[i - 1, l] > 0:                                   # i in Omega_l
                p[l, i] = 2.0 * PHI5[i - 1, l] / G[l]                # Theorems 6, 8
                eh[l, i] = mm[l][i] / (K[l] * p[l, i])
    est = np.zeros(22)
    var = np.zeros(22)
    lam = np.zeros((2, 22))     # a^(l)_i: lambda^(l)_i, 1 (single source) or 0
    plug = np.zeros(22)
    for i in range(1, 22):
        if i == 2:
            continue
        src = [l for l in range(2) if avail[l] and PHI5[i - 1, l] > 0]
        if not src:
            continue
        if len(src) == 1:
            l = src[0]
            e = eh[l, i] if eta is None else float(eta[i])
            plug[i] = e
            est[i] = eh[l, i]
            var[i] = e / K[l] * (1.0 / p[l, i] - e)                  # Theorems 7, 9
            lam[l, i] = 1.0
            continue
        if eta is None:
            e = (m1[i] + m2[i]) / (K1 * p[0, i] + K2 * p[1, i])      # pooled plug-in
        else:
            e = float(eta[i])
        plug[i] = e
        V1 = max(e / K1 * (1.0 / p[0, i] - e), 0.0)
        V2 = max(e / K2 * (1.0 / p[1, i] - e), 0.0)
        if V1 + V2 > 0.0:
            lam[0, i] = V2 / (V1 + V2)                               # lambda^(1)_i
            lam[1, i] = V1 / (V1 + V2)                               # lambda^(2)_i
            var[i] = V1 * V2 / (V1 + V2)                             # Theorem 10
        else:
            lam[0, i] = lam[1, i] = 0.5
            var[i] = 0.0
        est[i] = lam[0, i] * eh[0, i] + lam[1, i] * eh[1, i]         # eq. (mixestimator)
    # Cov(eta_i, eta_j) = -plug_i plug_j sum_l a^(l)_i a^(l)_j / K_l  (Theorem 10)
    cov = np.zeros((22, 22))
    for l in range(2):
        if avail[l]:
            a = lam[l] * plug
            cov -= np.outer(a, a) / K[l]
    np.fill_diagonal(cov, 0.0)
    # eta_2 = Lambda_4 - sum_{Omega_3*} phi^(3)_i eta_i  (Sec. 5.1.3)
    omega3 = [i for i in range(1, 22) if i != 2 and PHI5[i - 1, 2] > 0]
    s = 0.0
    for i in omega3:
        s += PHI5[i - 1, 2] * est[i]
    est[2] = float(Lambda4) - s
    v2 = 0.0
    for i in omega3:
        v2 += PHI5[i - 1, 2] ** 2 * var[i]
    for i in omega3:
        for j in omega3:
            if i != j:
                v2 += PHI5[i - 1, 2] * PHI5[j - 1, 2] * cov[i, j]
    var[2] = v2
    for i in range(22):
        cov[i, i] = var[i]
    # eta_2 is linear in the others: Cov(eta_2, eta_j) = -sum phi^(3)_i Cov(eta_i, eta_j)
    for j in range(1, 22):
        if j != 2:
            c2 = 0.0
            for i in omega3:
                c2 -= PHI5[i - 1, 2] * cov[i, j]
            cov[2, j] = cov[j, 2] = c2
    return {"k": 5, "K": (K1, K2), "est": est, "var": var, "lam": lam, "eta1": eh[0], "eta2": eh[1],
            "p": p, "plug": plug, "cov": cov, "conc": concentrations(est, 21)}
