"""Pins of the oracle's building blocks against things other than itself (CPU).

* SplitMix64 against its published reference outputs (tests/golden), and the
  word schedule against the generator's sequence.
* Philox4x32-10 against an independent implementation (Triton's, run by its
  CPU interpreter in a child process) on fixed and random counters and keys,
  and its word schedule against the block layout it defines.
* Alias tables: exact integer mass identity (each item gets w_j / W).
* Vertex weights Gamma, Gamma^(1), Gamma^(2), Lambda_3, Lambda_4 against
  brute-force counts of the draw sequences / subgraphs they stand for
  (Table 1, Sec. 4.1.1, Sec. 5.1.1, Sec. 5.1.2, eq. (2)).
* The classifier against networkx isomorphism for all masks (Table 2).
* The identities Lambda_3 = sum phi^(2) n_i (eq. 2) and Lambda_4 = sum phi^(3)
  eta_i (Sec. 5.1.3) on exact ESU counts, and ESU against all-subset scans.
"""
from __future__ import annotations

import itertools
import os

import numpy as np
import pytest

import oracle
import synth
from helpers import adjacency_sets, brute_force_cis, class_counts, mask_classes, phi4, table2

TWO64 = 1 << 64


# ------------------------------------------------------------ Philox4x32 --
_TRITON_PHILOX = r"""
import json, sys
import numpy as np
import torch, triton, triton.language as tl

@triton.jit
def k(seed_ptr, c_ptr, out_ptr, N: tl.constexpr):
    i = tl.arange(0, N)
    seed = tl.load(seed_ptr + i)
    a, b, c, d = tl.philox(seed, tl.load(c_ptr + 4 * i), tl.load(c_ptr + 4 * i + 1), tl.load(c_ptr + 4 * i + 2),
                           tl.load(c_ptr + 4 * i + 3), n_rounds=10)
    tl.store(out_ptr + 4 * i, a)
    tl.store(out_ptr + 4 * i + 1, b)
    tl.store(out_ptr + 4 * i + 2, c)
    tl.store(out_ptr + 4 * i + 3, d)

cases = json.load(sys.stdin)
n = len(cases)
seed = torch.tensor(np.array([kk[0] | (kk[1] << 32) for _, kk in cases], dtype=np.uint64))
ctr = torch.tensor(np.array([x for c, _ in cases for x in c], dtype=np.uint32))
out = torch.zeros(4 * n, dtype=torch.uint32)
k[(1,)](seed, ctr, out, N=n)
print(json.dumps([int(x) for x in out.numpy().view(np.uint32)]))
"""


def test_philox_matches_an_independent_implementation():
    """The oracle's Philox4x32-10 against triton.language.philox (10 rounds,
    key = the seed's low and high halves), evaluated on the CPU by Triton's
    interpreter in a child process."""
    import json
    import subprocess
    import sys
    pytest.importorskip("triton")
    rng = np.random.default_rng(2024)
    cases = [([0, 0, 0, 0], [0, 0]), ([0xFFFFFFFF] * 4, [0xFFFFFFFF] * 2), ([1, 0, 0, 0], [0, 0]),
             ([0, 0, 0, 1], [0, 1])]
    cases += [([int(x) for x in rng.integers(0, 2**32, 4)], [int(x) for x in rng.integers(0, 2**32, 2)])
              for _ in range(60)]          # 64 lanes: a power of two for tl.arange
    env = dict(os.environ, TRITON_INTERPRET="1")
    r = subprocess.run([sys.executable, "-c", _TRITON_PHILOX], input=json.dumps(cases), capture_output=True,
                       text=True, env=env, timeout=600)
    assert r.returncode == 0, r.stderr[-3000:]
    ref = json.loads(r.stdout.strip().splitlines()[-1])
    got = [x for c, kk in cases for x in oracle.philox4x32(c, kk)]
    assert got == ref


def test_philox_word_schedule_is_the_block_layout():
    """Words 2b and 2b+1 of sample s of method t are block (s lo, s hi, t, b)
    under the key (seed lo, seed hi), low output first."""
    seed, s, t = 0x0123456789ABCDEF, (7 << 32) + 99, 2
    w = oracle.sample_words(t, seed, s, 16, rng=oracle.PHILOX4X32)
    key = [seed & 0xFFFFFFFF, seed >> 32]
    for b in range(8):
        o = oracle.philox4x32([s & 0xFFFFFFFF, s >> 32, t, b], key)
        assert w[2 * b] == o[0] | (o[1] << 32)
        assert w[2 * b + 1] == o[2] | (o[3] << 32)
    # different methods and samples never share a block
    assert oracle.sample_words(1, seed, s, 2, rng=oracle.PHILOX4X32) != w[:2]
    assert oracle.sample_words(t, seed, s + 1, 2, rng=oracle.PHILOX4X32) != w[:2]


def test_philox_words_are_uniform():
    """Chi-square of the top four bits of 2^15 words (16 cells)."""
    counts = np.zeros(16)
    for s in range(2048):
        for x in oracle.sample_words(0, 77, s, 16, rng=oracle.PHILOX4X32):
            counts[x >> 60] += 1
    e = counts.sum() / 16
    chi2 = float(((counts - e) ** 2 / e).sum())
    assert chi2 < 45.0          # chi^2_15 exceeds 45 with probability < 1e-4


def test_philox_drives_the_samplers_unbiasedly():
    """Estimates under Philox words: the mean over 120 seeds is within 4.5
    sigma / sqrt(R) of the exact ESU counts (Theorems 3 and 10)."""
    import json
    gold = json.load(open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "esu_counts.json")))
    rp, col = synth.chung_lu(200, 2.3, 6.0, 30.0, seed=7)
    g = oracle.OracleGraph(rp, col)
    R = 120
    for k, key, budget in ((4, "esu4", 20_000), (5, "esu5", 20_000)):
        eta = np.array(gold["cl_n200"][key], dtype=np.float64)
        ref = g.estimate(k, budget, seed=0, eta=eta)
        est = np.array([g.estimate(k, budget, seed=900 + s, rng=oracle.PHILOX4X32)["est"] for s in range(R)])
        for i in range(1, 7 if k == 4 else 22):
            if i == 2 or eta[i] == 0:
                continue
            assert abs(est[:, i].mean() - eta[i]) < 4.5 * np.sqrt(ref["var"][i] / R) + 0.02 * eta[i] * (k == 5), (k, i)
    # the generator matters: the same seed gives other samples than SplitMix64
    assert not np.array_equal(g.run(oracle.T5, 3, 1000), g.run(oracle.T5, 3, 1000, rng=oracle.PHILOX4X32))


# -------------------------------------------------------------- SplitMix64 --
def _splitmix_golden():
    out = {}
    for line in open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "splitmix64.txt")):
        if line.strip() and not line.startswith("#"):
            kind, *vals = line.split()
            out[kind] = [int(v) for v in vals]
    return out


def test_splitmix_reference_outputs():
    seed, *ref = _splitmix_golden()["outputs"]
    assert [oracle.splitmix64(seed, k) for k in range(1, len(ref) + 1)] == ref


def test_splitmix_reference_buckets():
    seed, count, *ref = _splitmix_golden()["buckets"]
    counts = [0] * 5
    for k in range(1, count + 1):
        counts[oracle.splitmix64(seed, k) * 5 >> 64] += 1
    assert counts == ref


def test_word_schedule_follows_the_sequence():
    """Sample 0 of method 0 reads the generator's first outputs; sample s of
    method t starts 16 (4 s + t) outputs in, without overlap."""
    seed, *ref = _splitmix_golden()["outputs"]
    assert oracle.sample_words(0, seed, 0, len(ref)) == ref
    w = oracle.sample_words(2, seed, 3, 16)
    assert w[0] == oracle.splitmix64(seed, (4 * 3 + 2) * 16 + 1)
    seen = set()
    for s in range(4):
        for t in range(4):
            ws = oracle.sample_words(t, seed, s, 16)
            assert not seen & set(ws)
            seen |= set(ws)


# ------------------------------------------------------------------- alias --
def alias_mass_ok(w, thr, alias):
    m = len(w)
    W = sum(w)
    mass = [0] * m
    for j in range(m):
        assert 0 <= thr[j] <= W
        mass[j] += thr[j]
        if alias[j] != j:
            mass[alias[j]] += W - thr[j]
        else:
            assert thr[j] == W or W == 0
    for j in range(m):
        assert mass[j] == w[j] * m, (j, mass[j], w[j] * m)
        if w[j] == 0:
            assert all(alias[i] != j or i == j for i in range(m))


@pytest.mark.parametrize("case", range(12))
def test_alias_mass_identity(case):
    rng = np.random.default_rng(case)
    m = int(rng.integers(1, 300))
    kind = case % 4
    if kind == 0:
        w = [int(x) for x in rng.integers(0, 50, size=m)]
    elif kind == 1:   # huge 128-bit weights
        w = [int(rng.integers(0, 2**62)) * int(rng.integers(0, 2**40)) for _ in range(m)]
    elif kind == 2:   # equal weights: every column full
        w = [7] * m
    else:             # one dominant weight and many zeros
        w = [0] * m
        w[int(rng.integers(0, m))] = 10**20
        w[int(rng.integers(0, m))] += 3
    if sum(w) == 0:
        w[0] = 1
    thr, alias = oracle.alias_build(w)
    alias_mass_ok(w, thr, alias)


def test_alias_all_zero_weights():
    thr, alias = oracle.alias_build([0, 0, 0])
    assert thr == [0, 0, 0] and alias == [0, 1, 2]


def level_weights(vt, gam):
    """(heavy vertices, light vertices, W_H, W_L) of a two-level table."""
    nh = vt["nh"]
    heavy = [int(v) for v in vt["self"][:nh]]
    light = [int(v) for v in vt["self"][nh:]]
    return heavy, light, sum(gam[v] for v in heavy), sum(gam[v] for v in light)


@pytest.mark.parametrize("vsplit", [oracle.ONE_LEVEL, oracle.VSPLIT, 8, 3])
def test_vertex_tables_follow_their_definition(vsplit):
    """The two-level vertex tables: heavy vertices are exactly those with
    w_v 2^split >= W (ascending ids, then the light ones ascending); each
    level's table gives every vertex exactly its weight's share of the level
    (the alias mass identity); thresholds are floor(thr 2^64 / W_level); the
    light level's bound is floor(W_L 2^64 / W).  So a draw returns v with
    probability w_v / W up to the 2^-64 quantisation of each word."""
    rp, col = synth.workload("cl_n2k")
    g = oracle.OracleGraph(rp, col, vsplit=vsplit)
    deg, S, Q, gam = g.vertex()
    for which in range(3):
        vt = g.vertex_table(which)
        W = g.Gamma[which]
        heavy, light, WH, WL = level_weights(vt, gam[which])
        one = vsplit == oracle.ONE_LEVEL
        assert heavy == [v for v in range(g.n) if not one and gam[which][v] * (1 << vsplit) >= W]
        assert light == [v for v in range(g.n) if one or gam[which][v] * (1 << vsplit) < W]
        assert len(heavy) <= 1 << vsplit and WH + WL == W
        assert vt["TL"] == (min(WL * TWO64 // W, TWO64 - 1) if heavy else 0)
        nh = vt["nh"]
        for base, members, Wl in ((0, heavy, WH), (nh, light, WL)):
            m = len(members)
            if m == 0:
                continue
            pos = {v: i for i, v in enumerate(members)}
            thr = vt["thr"][base:base + m]
            alias = [pos[int(a)] for a in vt["alias"][base:base + m]]
            alias_mass_ok([gam[which][v] for v in members], thr, alias)
            for i in range(0, m, 7):
                assert int(vt["T"][base + i]) == (min(thr[i] * TWO64 // Wl, TWO64 - 1) if Wl else 0)
    if vsplit == oracle.ONE_LEVEL:   # one table over all vertices in id order
        assert all(list(g.vertex_table(l)["self"]) == list(range(g.n)) for l in range(3))
    if vsplit == 8:   # both levels hold mass
        assert all(0 < g.vertex_table(l)["nh"] <= 256 and g.vertex_table(l)["TL"] > 0 for l in range(3))
    if vsplit == 3:   # no vertex holds an eighth of Gamma or Gamma^(2): one light level only
        assert g.vertex_table(0)["nh"] == 0 and g.vertex_table(1)["nh"] > 0


def test_tables_of_workload_have_exact_mass():
    rp, col = synth.workload("cl_n2k")
    g = oracle.OracleGraph(rp, col)
    deg, S, Q, gam = g.vertex()
    gthr, galias, acc = g.sigma_table()
    for v in range(0, g.n, 13):
        o, d = int(rp[v]), int(rp[v + 1] - rp[v])
        w = [int(deg[int(x)]) - 1 for x in col[o:o + d]]
        if d:
            alias_mass_ok(w, [int(x) for x in gthr[o:o + d]], [int(x) for x in galias[o:o + d]])
            assert [int(x) for x in acc[o:o + d]] == list(itertools.accumulate([0] + w[:-1]))


# ----------------------------------------------------------------- weights --
def brute_weights(rp, col):
    """Count the draw sequences each weight stands for, by enumeration."""
    adj = adjacency_sets(rp, col)
    n = len(adj)
    G = G1 = G2 = 0
    for v in range(n):
        Nv = sorted(adj[v])
        for u in Nv:
            for w in Nv:
                if w == u:
                    continue
                for r in adj[u]:
                    if r != v:
                        G += 1              # (v, u, w in N_v-{u}, r in N_u-{v})
                for r in Nv:
                    if r in (u, w):
                        continue
                    for t in adj[u]:
                        if t != v:
                            G1 += 1         # T-5 sequences: w, r ordered distinct
                for r in adj[u]:
                    if r == v:
                        continue
                    for t in adj[w]:
                        if t != v:
                            G2 += 1         # Path-5 sequences (u, w ordered, distinct)
    L3 = sum(1 for v in range(n) for _ in itertools.combinations(adj[v], 3))
    L4 = sum(1 for v in range(n) for _ in itertools.combinations(adj[v], 4))
    return G, G1, G2, L3, L4


@pytest.mark.parametrize("seed", [1, 2, 3, 4])
def test_weights_count_draw_sequences(seed):
    rp, col = synth.gnp(11, 0.4, seed)
    g = oracle.OracleGraph(rp, col)
    G, G1, G2, L3, L4 = brute_weights(rp, col)
    # Gamma counts ordered (v,u,w,r) sequences; Gamma^(1) counts (v,u,w,r,t)
    # with (w, r) an ordered pair, i.e. 2x the unordered choice the
    # probability 1/((d_v-1)(d_v-2)) refers to; Gamma^(2) counts ordered (u, w).
    assert g.Gamma[0] == G
    assert g.Gamma[1] == G1
    assert g.Gamma[2] == G2
    assert g.Lambda3 == L3
    assert g.Lambda4 == L4


def test_weights_on_star_cycle_complete():
    g = oracle.OracleGraph(*synth.star(6))
    assert g.Gamma == [0, 0, 0] and g.Lambda3 == 20 and g.Lambda4 == 15
    g = oracle.OracleGraph(*synth.cycle(9))
    assert g.Gamma == [18, 0, 18] and g.Lambda3 == 0
    n = 7
    g = oracle.OracleGraph(*synth.complete(n))
    d = n - 1
    assert g.Gamma[0] == n * (d - 1) * d * (d - 1)


# ---------------------------------------------------------------- classify --
@pytest.mark.parametrize("k", [4, 5])
def test_classifier_matches_networkx_on_all_masks(k):
    ref = mask_classes(k)
    for mask in range(len(ref)):
        assert oracle.classify(k, mask) == ref[mask], mask


def test_table2_signatures_are_unique_and_complete():
    from helpers import motif_atlas
    at5 = motif_atlas(5)
    assert len(at5) == 21
    assert sorted(c for _, _, c in at5) == list(range(1, 22))
    at4 = motif_atlas(4)
    assert sorted(c for _, _, c in at4) == list(range(1, 7))


# -------------------------------------------------------------- identities --
@pytest.mark.parametrize("seed", [5, 6])
def test_esu_matches_all_subsets_and_identities(seed):
    rp, col = synth.gnp(12, 0.45, seed)
    g = oracle.OracleGraph(rp, col)
    for k in (4, 5):
        ref = class_counts(brute_force_cis(rp, col, k), 22)
        got = g.esu(k).astype(np.int64)
        assert (got == ref).all(), (k, got, ref)
    n4 = g.esu(4).astype(np.int64)
    p4 = phi4()
    # eq. (2): Lambda_3 = sum_i phi^(2)_i n_i
    assert g.Lambda3 == sum(p4[i][1] * int(n4[i]) for i in range(1, 7))
    n5 = g.esu(5).astype(np.int64)
    t2 = table2()
    # Sec. 5.1.3: Lambda_4 = sum_i phi^(3)_i eta_i
    assert g.Lambda4 == sum(t2[i][2] * int(n5[i]) for i in range(1, 22))


def test_identities_on_power_law_graph():
    rp, col = synth.chung_lu(300, 2.3, 6.0, 40.0, seed=3)
    g = oracle.OracleGraph(rp, col)
    n4 = g.esu(4).astype(np.int64)
    p4 = phi4()
    assert g.Lambda3 == sum(p4[i][1] * int(n4[i]) for i in range(1, 7))
    n5 = g.esu(5).astype(np.int64)
    t2 = table2()
    assert g.Lambda4 == sum(t2[i][2] * int(n5[i]) for i in range(1, 22))


def test_default_vertex_splits():
    """The default level split: one level below 2^14 vertices, split 12 up to
    2^20, split 20 from there; the MOSS-4Min table one level below 2^20."""
    assert [oracle.default_split(n) for n in (1, (1 << 14) - 1, 1 << 14, (1 << 20) - 1, 1 << 20)] == \
        [oracle.ONE_LEVEL, oracle.ONE_LEVEL, oracle.VSPLIT_MID, oracle.VSPLIT_MID, oracle.VSPLIT]
    assert [oracle.default_split_min(n) for n in (1 << 14, (1 << 20) - 1, 1 << 20)] == \
        [oracle.ONE_LEVEL, oracle.ONE_LEVEL, oracle.VSPLIT]
    rp, col = synth.chung_lu(1 << 14, 2.2, 8.0, 200.0, seed=3)
    g = oracle.OracleGraph(rp, col)
    assert (g.vsplit, g.vsplit_min) == (oracle.VSPLIT_MID, oracle.ONE_LEVEL)
    assert all(g.vertex_table(l)["nh"] > 0 for l in range(3))
    g.build_min()
    assert g.vertex_table(3)["nh"] == 0
    assert oracle.OracleGraph(rp, col, vsplit=9).vsplit_min == 9
