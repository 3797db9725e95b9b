"""The numpy statement of MOSS_ORDER_DEGREE (helpers.degree_order) that the
GPU tests compare the library's renumbering with, pinned to its definition:
the key's values from the formula by hand, and on small graphs a plain
Python renumbering (sort by key then id, relabel, sort every list)."""
from __future__ import annotations

import numpy as np
import pytest

import synth
from helpers import degree_order, order_key


def test_key_values():
    # d < 16: d itself; then 16 + 4 (L - 5) + the two bits below the leading one
    hand = {0: 0, 1: 1, 15: 15, 16: 16, 19: 16, 20: 17, 24: 18, 28: 19, 31: 19, 32: 20, 40: 21, 47: 21,
            48: 22, 63: 23, 64: 24, 1000: 16 + 4 * 5 + 3, 1024: 16 + 4 * 6, (1 << 31) - 1: 16 + 4 * 26 + 3,
            1 << 31: 16 + 4 * 27, (1 << 32) - 1: 127}
    got = order_key(np.array(list(hand), dtype=np.int64))
    assert got.tolist() == list(hand.values())


def test_key_is_monotone_in_degree():
    d = np.arange(0, 1 << 20, dtype=np.int64)
    k = order_key(d)
    assert (np.diff(k) >= 0).all() and k[-1] == 16 + 4 * 15 + 3


def plain_renumbering(rp, col):
    n = len(rp) - 1
    deg = [int(rp[v + 1] - rp[v]) for v in range(n)]

    def key(d):
        if d < 16:
            return d
        L = d.bit_length()
        return 16 + 4 * (L - 5) + ((d >> (L - 3)) & 3)

    order = sorted(range(n), key=lambda v: (-key(deg[v]), v))
    inv = {v: i for i, v in enumerate(order)}
    lists = [sorted(inv[int(u)] for u in col[rp[v]:rp[v + 1]]) for v in order]
    nrp = np.cumsum([0] + [len(l) for l in lists])
    return np.array(order), nrp, np.array([x for l in lists for x in l], dtype=np.int64)


@pytest.mark.parametrize("graph", [
    lambda: synth.chung_lu(3000, 2.1, 9.0, 600.0, seed=4),
    lambda: synth.star(40),
    lambda: synth.from_edges(37, [(2, 5), (5, 7), (2, 7), (30, 36), (7, 30)]),
    lambda: synth.rgg(500, 10.0, seed=2),
])
def test_degree_order_matches_plain_renumbering(graph):
    rp, col = graph()
    order, nrp, ncol = degree_order(rp, col)
    o2, r2, c2 = plain_renumbering(rp, col)
    assert np.array_equal(order, o2)
    assert np.array_equal(nrp.astype(np.int64), r2)
    assert np.array_equal(ncol.astype(np.int64), c2)
    # an isomorphism: edge (a, b) of the input is (inv a, inv b) of the output
    n = len(rp) - 1
    inv = np.empty(n, dtype=np.int64)
    inv[order.astype(np.int64)] = np.arange(n)
    src = np.repeat(np.arange(n), np.diff(rp.astype(np.int64)))
    e_in = {(int(inv[a]), int(inv[b])) for a, b in zip(src, col)}
    nsrc = np.repeat(np.arange(n), np.diff(nrp.astype(np.int64)))
    assert e_in == {(int(a), int(b)) for a, b in zip(nsrc, ncol)}
