"""The library's host-built classification tables (no GPU needed), against
independent definitions written here: the motif class of every 4- and
5-vertex edge mask by networkx isomorphism (Sec. 4.1.2, Table 2), and c(s)
of MOSS-4Min (Sec. 4.2) for every 4-vertex mask and every total order of
its vertices by brute force over the ordered 3-paths."""
from __future__ import annotations

import itertools

import pytest

import paper_1509_08089_gb300 as moss
from helpers import nx_class

PAIRS4 = [(0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3)]
PAIRS5 = [(a, b) for a in range(5) for b in range(a + 1, 5)]


@pytest.fixture(scope="module")
def tables():
    return moss.moss_class_tables()


@pytest.mark.parametrize("k", [4, 5])
def test_class_tables_match_networkx(tables, k):
    lut = tables[0] if k == 4 else tables[1]
    pairs = PAIRS4 if k == 4 else PAIRS5
    for mask in range(1 << len(pairs)):
        edges = [pairs[b] for b in range(len(pairs)) if mask >> b & 1]
        assert int(lut[mask]) == nx_class(k, edges), (k, mask)


def brute_force_c(edges: set, above) -> int:
    """Ordered 3-paths p0-p1-p2-p3 with p0 above p2 and p3 above p1, halved
    (a path and its reverse satisfy the condition together)."""
    count = 0
    for p in itertools.permutations(range(4)):
        if all(frozenset((p[i], p[i + 1])) in edges for i in range(3)):
            count += above(p[0], p[2]) and above(p[3], p[1])
    assert count % 2 == 0
    return count // 2


def test_centred_path_table_matches_brute_force(tables):
    class4, cc = tables[0], tables[2]
    counted = {3, 5, 6}            # 4-cycle, diamond, 4-clique
    seen = {3: set(), 5: set(), 6: set()}
    for mask in range(64):
        edges = {frozenset(PAIRS4[b]) for b in range(6) if mask >> b & 1}
        cls = int(class4[mask])
        for rank in itertools.permutations(range(4)):   # rank[x]: position of role x, 0 = highest
            above = lambda a, b, r=rank: r[a] < r[b]
            bits = sum(1 << b for b, (x, y) in enumerate(PAIRS4) if above(x, y))
            got = int(cc[mask << 6 | bits])
            if cls in counted:
                want = brute_force_c(edges, above)
                assert got == want, (mask, rank, got, want)
                seen[cls].add(got)
            else:
                assert got == 0, (mask, rank)
    # Sec. 4.2 (with the corrected Theorem 4): c = 1 for every 4-cycle, 3 for
    # every 4-clique, and 1, 2 or 3 for a diamond depending on the order
    assert seen == {3: {1}, 5: {1, 2, 3}, 6: {3}}
