"""Pins of the oracle's BVC-PLL (Alg. 4, Sec. 4.2): for every batch size the
labels are Def. 2's (the paper's correctness remark after Alg. 4), a batch
of one behaves as PLL, and the messages BVC-PLL sends equal the distance
checks PLL runs minus the roots' own (Sec. 4.3: the same hubs reach the same
vertices, and each message is one check)."""
import numpy as np
import pytest

import oracle as O
from paper_1906_12018_gb300 import graphs as G

from test_oracle import tiny_graphs


def same(a, b):
    return np.array_equal(a.off, b.off) and np.array_equal(a.hub, b.hub) and np.array_equal(a.dist, b.dist)


@pytest.mark.parametrize("name,g", tiny_graphs(), ids=lambda x: x if isinstance(x, str) else "")
def test_every_batch_size_gives_def2(name, g):
    rng = np.random.default_rng(3)
    for order in (G.degree_order(g), rng.permutation(g.n).astype(np.int32)):
        ref = O.chhl(g.off, g.col, order)
        for B in sorted({1, 2, 3, 7, max(1, g.n)}):
            assert same(O.bvcpll(g.off, g.col, order, B), ref), (name, B)


@pytest.mark.parametrize("B", [1, 16, 256, 1024, 4096])
def test_rmat12_batches(B):
    g = G.workload("rmat12")
    order = G.degree_order(g)
    P = O.pll(g.off, g.col, order)
    L = O.bvcpll(g.off, g.col, order, B)
    assert same(L, P)
    assert L.checks == P.checks - g.n      # the roots' own (u, 0) is no message


def test_chung_lu_with_isolated_vertices():
    g = G.chung_lu_graph(3000, 8.0, 2.1, 9)
    order = G.degree_order(g)
    P = O.pll(g.off, g.col, order)
    for B in (1, 100, 3000):
        L = O.bvcpll(g.off, g.col, order, B)
        assert same(L, P) and L.checks == P.checks - g.n
