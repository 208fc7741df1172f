"""The seeded synthetic inputs that stand in for the paper's graphs: the
properties the input recipe states (symmetric simple CSR with ascending
rows, the LCC connected, the recorded sizes, the batch's size range, the
degree order's tie rule, seeding)."""
import numpy as np
import pytest

import oracle as O
from paper_1906_12018_gb300 import graphs as G


def assert_simple_symmetric(g):
    src = np.repeat(np.arange(g.n), np.diff(g.off))
    assert np.all(g.col >= 0) and np.all(g.col < g.n)
    assert not np.any(src == g.col)                                   # no self-loops
    for v in range(0, g.n, max(1, g.n // 257)):                       # rows strictly ascending (sampled)
        r = g.col[g.off[v]:g.off[v + 1]]
        assert np.all(np.diff(r) > 0)
    fwd = np.sort(src.astype(np.int64) * g.n + g.col)
    rev = np.sort(g.col.astype(np.int64) * g.n + src)
    assert np.array_equal(fwd, rev)                                   # (u,v) present iff (v,u)


def test_rmat12_recipe():
    g = G.workload("rmat12")
    assert (g.n, g.m) == (3008, 26705)
    assert_simple_symmetric(g)
    assert np.all(O.bfs(g.off, g.col, 0) >= 0)                        # the LCC is connected
    assert np.array_equal(g.col, G.workload("rmat12").col)            # seeded


def test_chung_lu_recipe():
    g = G.chung_lu_graph(1 << 14, 16.0, 2.1, 2)
    assert g.n == 1 << 14
    assert_simple_symmetric(g)
    deg = np.diff(g.off)
    assert 0 < deg.mean() < 16.0                                      # below the target after dedup
    assert np.argmax(deg) < 16                                        # weights fall with the index
    assert np.any(deg == 0)                                           # isolated vertices are kept
    assert not np.array_equal(deg, np.diff(G.chung_lu_graph(1 << 14, 16.0, 2.1, 3).off))


def test_batch_sizes_and_kinds():
    sizes = np.array([G.small_graph_size(i) for i in range(2000)])
    assert sizes.min() >= 1024 and sizes.max() <= 65536
    assert np.median(np.log2(sizes)) == pytest.approx(13.0, abs=0.3)  # log-uniform on [10, 16]
    for i in (0, 1):
        g = G.small_graph(i)
        assert_simple_symmetric(g)
        if i % 2 == 0:                                                # R-MAT + LCC: connected
            assert np.all(O.bfs(g.off, g.col, 0) >= 0)
        else:                                                         # Chung-Lu: all vertices kept
            assert g.n == sizes[i]


def test_degree_order_rule():
    g = G.workload("rmat12")
    order = G.degree_order(g)
    deg = np.diff(g.off)[order]
    assert sorted(order.tolist()) == list(range(g.n))
    assert np.all(np.diff(deg) <= 0)                                  # degree descending
    ties = np.diff(deg) == 0
    assert np.all(np.diff(order)[ties] > 0)                           # ties by smaller id


def test_query_pairs():
    p = G.uniform_pairs(1000, 5000, 1)
    assert p.shape == (5000, 2) and p.min() >= 0 and p.max() < 1000
    assert np.array_equal(p, G.uniform_pairs(1000, 5000, 1))
    assert abs(p.mean() - 499.5) < 15


def test_directed_recipe():
    g = G.rmat_digraph(10, 16, 3)
    src = np.repeat(np.arange(g.n), np.diff(g.off))
    key = src.astype(np.int64) * g.n + g.col
    assert not np.any(src == g.col) and len(np.unique(key)) == len(key)  # no self-loops, no duplicate arcs
    srci = np.repeat(np.arange(g.n), np.diff(g.off_in))
    assert np.array_equal(np.sort(key), np.sort(g.col_in.astype(np.int64) * g.n + srci))  # the transpose
