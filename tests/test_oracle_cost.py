"""Pins of the oracle's positive distance-check cost counters (Sec. 4.3, the
theorem on positive distance checks and its figure): the figure's example
of nine hubs of one vertex arriving in three distance groups of three
(36 label reads under PLL, 27 under VC-PLL), and on any graph the proof's
closed forms computed from the output labels: under PLL a vertex with n
hubs besides itself reads n(n-1)/2 labels, under VC-PLL
n(n-1)/2 - sum_i n_i(n_i-1)/2 over its groups of equal distance."""
import numpy as np
import pytest

import oracle as O
from paper_1906_12018_gb300 import graphs as G


def three_paths():
    """v = 0 with three disjoint paths v-a-d-g, v-b-e-h, v-c-f-i (a..i =
    1..9); ranks g, h, i, d, e, f, a, b, c, v: every one of the nine is a
    hub of v (each outranks the rest of its path to v), at distance 3, 2, 1."""
    edges = [(0, 1), (0, 2), (0, 3), (1, 4), (2, 5), (3, 6), (4, 7), (5, 8), (6, 9)]
    s = [a for a, b in edges] + [b for a, b in edges]
    t = [b for a, b in edges] + [a for a, b in edges]
    g = G.clean_csr(10, np.array(s), np.array(t))
    order = np.array([7, 8, 9, 4, 5, 6, 1, 2, 3, 0], dtype=np.int32)
    return g, order


def test_figure_example_36_against_27():
    g, order = three_paths()
    P = O.pll(g.off, g.col, order)
    V = O.vcpll(g.off, g.col, order)
    h, d = P.row(0)
    assert len(h) == 10 and sorted(d.tolist()) == [0, 1, 1, 1, 2, 2, 2, 3, 3, 3]
    assert P.cost[0] == 36          # 0 + 1 + ... + 8
    assert V.cost[0] == 27          # 3 x 3 + 3 x 6
    assert np.array_equal(P.hub, V.hub) and np.array_equal(P.dist, V.dist)


def closed_forms(L):
    pll, vc = np.zeros(L.n, np.int64), np.zeros(L.n, np.int64)
    for v in range(L.n):
        h, d = L.row(v)
        d = d[d > 0]                # v's own (v, 0) is not counted
        n = len(d)
        groups = np.bincount(d.astype(np.int64))
        pll[v] = n * (n - 1) // 2
        vc[v] = pll[v] - int(np.sum(groups * (groups - 1) // 2))
    return pll, vc


@pytest.mark.parametrize("graph", ["rmat10", "chunglu", "grid"])
def test_costs_equal_the_closed_forms(graph):
    if graph == "rmat10":
        g = G.rmat_graph(10, 8, 3)
    elif graph == "chunglu":
        g = G.chung_lu_graph(1500, 8.0, 2.1, 5)
    else:
        s = [r * 12 + c for r in range(12) for c in range(11)] + [r * 12 + c for r in range(11) for c in range(12)]
        t = [r * 12 + c + 1 for r in range(12) for c in range(11)] + [(r + 1) * 12 + c for r in range(11) for c in range(12)]
        g = G.clean_csr(144, np.array(s + t), np.array(t + s))
    order = G.degree_order(g)
    P = O.pll(g.off, g.col, order)
    V = O.vcpll(g.off, g.col, order)
    want_p, want_v = closed_forms(P)
    assert np.array_equal(P.cost, want_p)
    assert np.array_equal(V.cost, want_v)
    assert V.cost.sum() <= P.cost.sum()   # the theorem: never more than PLL
