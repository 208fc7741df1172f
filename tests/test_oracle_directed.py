"""Pins of the directed oracle (Sec. 5.1) against things other than itself:
Def. 2 for directed graphs re-derived from scipy's directed all-pairs
distances and the shortest-path sets, directed all-pairs distances for the
queries, closed forms for the directed path and cycle, invariants, and the
symmetric digraph equal to the undirected labeling."""
import numpy as np
import pytest

sp = pytest.importorskip("scipy.sparse")
from scipy.sparse.csgraph import shortest_path  # noqa: E402

import oracle as O  # noqa: E402
from paper_1906_12018_gb300 import graphs as G  # noqa: E402


def dapsp(g):
    """D[u, v] = d(u -> v) (inf when v is not reachable)."""
    n = g.n
    a = sp.csr_matrix((np.ones(g.arcs), g.col, g.off), shape=(n, n))
    return shortest_path(a, method="D", unweighted=True, directed=True)


def directed_labels_by_definition(g, order):
    """h in L_in(v) iff rank(h) is the minimum over P_hv = {w : d(h,w) + d(w,v)
    = d(h,v)}; h in L_out(v) iff rank(h) is the minimum over P_vh."""
    n = g.n
    D = dapsp(g)
    rank = np.empty(n, dtype=np.int64)
    rank[order] = np.arange(n)
    lin, lout = [], []
    for v in range(n):
        rin, rout = [], []
        for h in range(n):
            if np.isfinite(D[h, v]):
                on = np.isfinite(D[h]) & np.isfinite(D[:, v]) & (D[h] + D[:, v] == D[h, v])
                if rank[on].min() == rank[h]:
                    rin.append((int(rank[h]), int(D[h, v])))
            if np.isfinite(D[v, h]):
                on = np.isfinite(D[v]) & np.isfinite(D[:, h]) & (D[v] + D[:, h] == D[v, h])
                if rank[on].min() == rank[h]:
                    rout.append((int(rank[h]), int(D[v, h])))
        lin.append(sorted(rin))
        lout.append(sorted(rout))
    return lin, lout


def rows(L):
    return [list(zip(L.hub[L.off[v]:L.off[v + 1]].tolist(), L.dist[L.off[v]:L.off[v + 1]].tolist()))
            for v in range(L.n)]


def tiny_digraphs():
    rng = np.random.default_rng(11)
    out = []
    for n, p in [(1, 0.0), (2, 1.0), (6, 0.4), (9, 0.3), (14, 0.2), (20, 0.12), (24, 0.25)]:
        m = rng.random((n, n)) < p
        s, d = np.nonzero(m)
        out.append((f"er{n}-{p}", G.directed_csr(n, s, d)))
    out.append(("path8", G.directed_csr(8, np.arange(7), np.arange(1, 8))))
    out.append(("cycle9", G.directed_csr(9, np.arange(9), (np.arange(9) + 1) % 9)))
    # a DAG, a tournament, and two strongly connected parts joined one way
    s, d = np.nonzero(np.triu(rng.random((12, 12)) < 0.3, 1))
    out.append(("dag12", G.directed_csr(12, s, d)))
    t = rng.random((7, 7)) < 0.5
    s, d = np.nonzero(np.triu(t, 1) | np.tril(~t.T, -1))
    out.append(("tournament7", G.directed_csr(7, s, d)))
    a = [(0, 1), (1, 2), (2, 0), (2, 3), (3, 4), (4, 5), (5, 3), (1, 4)]
    out.append(("two-scc", G.directed_csr(6, [x for x, _ in a], [y for _, y in a])))
    return out


def orders_for(g, rng):
    yield G.directed_degree_order(g)
    yield np.arange(g.n, dtype=np.int32)
    yield rng.permutation(g.n).astype(np.int32)


@pytest.mark.parametrize("name,g", tiny_digraphs(), ids=lambda x: x if isinstance(x, str) else "")
def test_directed_labels_match_apsp_definition(name, g):
    rng = np.random.default_rng(5)
    for order in orders_for(g, rng):
        lin, lout = directed_labels_by_definition(g, order)
        Ci, Co = O.chhl_directed(g.off, g.col, g.off_in, g.col_in, order)
        Pi, Po = O.pll_directed(g.off, g.col, g.off_in, g.col_in, order)
        assert rows(Ci) == lin and rows(Co) == lout, name
        assert rows(Pi) == lin and rows(Po) == lout, name


@pytest.mark.parametrize("name,g", tiny_digraphs(), ids=lambda x: x if isinstance(x, str) else "")
def test_directed_queries_equal_apsp(name, g):
    order = G.directed_degree_order(g)
    Li, Lo = O.pll_directed(g.off, g.col, g.off_in, g.col_in, order)
    D = dapsp(g)
    pairs = np.array([(s, t) for s in range(g.n) for t in range(g.n)], dtype=np.int32).reshape(-1, 2)
    got = O.query_directed(Lo, Li, pairs)
    want = np.where(np.isfinite(D[pairs[:, 0], pairs[:, 1]]), D[pairs[:, 0], pairs[:, 1]], -1).astype(np.int32)
    assert np.array_equal(got, want), name


def test_directed_path_and_cycle_closed_forms():
    n = 9
    ident = np.arange(n, dtype=np.int32)
    p = G.directed_csr(n, np.arange(n - 1), np.arange(1, n))
    Li, Lo = O.pll_directed(p.off, p.col, p.off_in, p.col_in, ident)
    assert rows(Li) == [[(h, v - h) for h in range(v + 1)] for v in range(n)]   # every earlier vertex reaches v
    assert rows(Lo) == [[(v, 0)] for v in range(n)]                              # v reaches only later ones
    c = G.directed_csr(n, np.arange(n), (np.arange(n) + 1) % n)
    Li, Lo = O.pll_directed(c.off, c.col, c.off_in, c.col_in, ident)
    assert rows(Li) == [[(h, v - h) for h in range(v + 1)] for v in range(n)]
    assert rows(Lo) == [[(0, 0)]] + [[(0, n - v), (v, 0)] for v in range(1, n)]  # v -> 0 wraps around
    assert Li.total + Lo.total == n * (n + 1) // 2 + 2 * n - 1


def test_symmetric_digraph_is_the_undirected_labeling():
    g = G.rmat_graph(9, 8, 2)
    order = G.degree_order(g)
    d = G.directed_csr(g.n, np.repeat(np.arange(g.n), np.diff(g.off)), g.col)
    Li, Lo = O.pll_directed(d.off, d.col, d.off_in, d.col_in, order)
    U = O.pll(g.off, g.col, order)
    for L in (Li, Lo):
        assert np.array_equal(L.off, U.off) and np.array_equal(L.hub, U.hub) and np.array_equal(L.dist, U.dist)


def test_directed_invariants_on_rmat():
    g = G.rmat_digraph(11, 8, 3)
    order = G.directed_degree_order(g)
    Li, Lo = O.pll_directed(g.off, g.col, g.off_in, g.col_in, order)
    rank = np.empty(g.n, dtype=np.int64)
    rank[order] = np.arange(g.n)
    rng = np.random.default_rng(1)
    for v in rng.choice(g.n, 40, replace=False):
        din = O.bfs(g.off_in, g.col_in, int(v))    # d(x -> v)
        dout = O.bfs(g.off, g.col, int(v))         # d(v -> x)
        for L, dd in ((Li, din), (Lo, dout)):
            h, d = L.row(v)
            assert np.all(np.diff(h.astype(np.int64)) > 0)             # sorted, unique
            assert h[-1] == rank[v] and d[-1] == 0                      # (v, 0) closes the row
            assert np.all(h.astype(np.int64) <= rank[v])                # hierarchy
            assert np.array_equal(d.astype(np.int32), dd[order[h]])     # exact distances
