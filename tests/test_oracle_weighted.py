"""Pins of the weighted oracle (Sec. 5.1; the PLL-with-Dijkstra baseline of
Sec. 6.4) against things other than itself: Def. 2 re-derived from scipy's
weighted all-pairs distances and the shortest-path sets, all-pairs distances
for the queries, the unweighted oracle (unit weights, and every edge of
weight w subdivided into w unit edges through vertices ranked last), scaling
of all weights, closed forms for weighted paths, hand-derived triangles, and
invariants."""
import numpy as np
import pytest

sp = pytest.importorskip("scipy.sparse")
from scipy.sparse.csgraph import shortest_path  # noqa: E402

import oracle as O  # noqa: E402
from paper_1906_12018_gb300 import graphs as G  # noqa: E402


def wgraph(n, edges):
    """Symmetric CSR and per-arc weights from undirected (u, v, w) triples."""
    es = {}
    for u, v, w in edges:
        es[(min(u, v), max(u, v))] = w
    src = [a for a, b in es] + [b for a, b in es]
    dst = [b for a, b in es] + [a for a, b in es]
    g = G.clean_csr(n, np.array(src, np.int64), np.array(dst, np.int64))
    wt = np.array([es[(min(u, v), max(u, v))] for u, v in zip(np.repeat(np.arange(n), np.diff(g.off)), g.col)],
                  dtype=np.uint8)
    return g, wt


def apsp(g, wt):
    a = sp.csr_matrix((wt.astype(np.float64), g.col, g.off), shape=(g.n, g.n))
    return shortest_path(a, method="D", directed=True)


def labels_by_definition(g, wt, order):
    """h in L(v) iff rank(h) is the minimum over P_hv = {w : d(h,w) + d(w,v)
    = d(h,v)}, the vertices of all shortest h-v paths."""
    D = apsp(g, wt)
    rank = np.empty(g.n, dtype=np.int64)
    rank[order] = np.arange(g.n)
    out = []
    for v in range(g.n):
        row = []
        for h in range(g.n):
            if np.isfinite(D[h, v]):
                on = np.isfinite(D[h]) & (D[h] + D[:, v] == D[h, v])
                if rank[on].min() == rank[h]:
                    row.append((int(rank[h]), int(D[h, v])))
        out.append(sorted(row))
    return out


def rows(L):
    return [list(zip(L.hub[L.off[v]:L.off[v + 1]].tolist(), L.dist[L.off[v]:L.off[v + 1]].tolist()))
            for v in range(L.n)]


def tiny_wgraphs():
    rng = np.random.default_rng(21)
    out = []
    for n, p, wmax in [(1, 0.0, 1), (2, 1.0, 3), (6, 0.5, 7), (9, 0.35, 7), (14, 0.25, 3), (20, 0.15, 7),
                       (24, 0.3, 2), (16, 0.4, 1)]:
        m = np.triu(rng.random((n, n)) < p, 1)
        s, d = np.nonzero(m)
        e = [(int(a), int(b), int(rng.integers(1, wmax + 1))) for a, b in zip(s, d)]
        out.append((f"er{n}-{p}-w{wmax}", *wgraph(n, e)))
    out.append(("path7", *wgraph(7, [(i, i + 1, 1 + (3 * i) % 5) for i in range(6)])))
    out.append(("cycle8", *wgraph(8, [(i, (i + 1) % 8, 1 + i % 3) for i in range(8)])))
    # equal-length alternatives everywhere (ties on the shortest paths)
    out.append(("grid3x4-w2", *wgraph(12, [(r * 4 + c, r * 4 + c + 1, 2) for r in range(3) for c in range(3)] +
                                      [(r * 4 + c, (r + 1) * 4 + c, 2) for r in range(2) for c in range(4)])))
    # heavy shortcut edges that lose to multi-hop paths
    out.append(("shortcuts", *wgraph(6, [(0, 1, 1), (1, 2, 1), (2, 3, 1), (0, 3, 7), (3, 4, 2), (0, 4, 4),
                                         (4, 5, 1), (1, 5, 6)])))
    return out


def orders_for(g, rng):
    yield G.degree_order(g)
    yield np.arange(g.n, dtype=np.int32)
    yield rng.permutation(g.n).astype(np.int32)


@pytest.mark.parametrize("name,g,wt", tiny_wgraphs(), ids=lambda x: x if isinstance(x, str) else "")
def test_weighted_labels_match_apsp_definition(name, g, wt):
    rng = np.random.default_rng(5)
    for order in orders_for(g, rng):
        want = labels_by_definition(g, wt, order)
        assert rows(O.pll_weighted(g.off, g.col, wt, order)) == want, name
        assert rows(O.chhl_weighted(g.off, g.col, wt, order)) == want, name


@pytest.mark.parametrize("name,g,wt", tiny_wgraphs(), ids=lambda x: x if isinstance(x, str) else "")
def test_weighted_queries_and_dijkstra_equal_apsp(name, g, wt):
    L = O.pll_weighted(g.off, g.col, wt, G.degree_order(g))
    D = apsp(g, wt)
    pairs = np.array([(s, t) for s in range(g.n) for t in range(g.n)], dtype=np.int32).reshape(-1, 2)
    want = np.where(np.isfinite(D[pairs[:, 0], pairs[:, 1]]), D[pairs[:, 0], pairs[:, 1]], -1).astype(np.int32)
    assert np.array_equal(O.query(L, pairs), want), name
    for s in range(min(g.n, 5)):
        assert np.array_equal(O.dijkstra(g.off, g.col, wt, s), want.reshape(g.n, g.n)[s]), name


def test_unit_weights_are_the_unweighted_labeling():
    g = G.rmat_graph(10, 8, 4)
    order = G.degree_order(g)
    W = O.pll_weighted(g.off, g.col, np.ones(g.col.shape[0], np.uint8), order)
    U = O.pll(g.off, g.col, order)
    assert np.array_equal(W.off, U.off) and np.array_equal(W.hub, U.hub) and np.array_equal(W.dist, U.dist)


def subdivide(g, wt):
    """Every edge {u, v} of weight w becomes a path of w unit edges through
    w - 1 new vertices (numbered from n on)."""
    n = g.n
    src = np.repeat(np.arange(n), np.diff(g.off))
    s_out, d_out = [], []
    nxt = n
    for u, v, w in zip(src.tolist(), g.col.tolist(), wt.tolist()):
        if u > v:
            continue
        chain = [u] + list(range(nxt, nxt + w - 1)) + [v]
        nxt += w - 1
        for a, b in zip(chain[:-1], chain[1:]):
            s_out += [a, b]
            d_out += [b, a]
    return G.clean_csr(nxt, np.array(s_out, np.int64), np.array(d_out, np.int64)), nxt


def test_subdivided_graph_gives_the_weighted_labeling():
    """Subdividing preserves the distances between original vertices and their
    shortest paths; the new vertices rank below every original one, so the
    highest-ranked vertex of each shortest path is unchanged and the rows of the
    original vertices are exactly the weighted labels (hub ranks below n)."""
    g = G.rmat_graph(8, 6, 7)
    wt = G.edge_weights(g, 1, 4, 9)
    order = G.degree_order(g)
    sg, N = subdivide(g, wt)
    sorder = np.concatenate([order, np.arange(g.n, N, dtype=np.int32)])
    U = O.pll(sg.off, sg.col, sorder)
    W = O.pll_weighted(g.off, g.col, wt, order)
    for v in range(g.n):
        h, d = U.row(v)
        hw, dw = W.row(v)
        assert np.all(h < g.n)
        assert np.array_equal(h, hw) and np.array_equal(d, dw), v


@pytest.mark.parametrize("k", [2, 3])
def test_scaling_all_weights_scales_the_distances(k):
    g = G.chung_lu_graph(600, 6.0, 2.3, 4)
    wt = G.edge_weights(g, 1, 7, 3)
    order = G.degree_order(g)
    A = O.pll_weighted(g.off, g.col, wt, order)
    B = O.pll_weighted(g.off, g.col, (wt * k).astype(np.uint8), order)
    assert np.array_equal(A.off, B.off) and np.array_equal(A.hub, B.hub)
    assert np.array_equal(A.dist.astype(np.int32) * k, B.dist.astype(np.int32))


def test_weighted_path_closed_form():
    w = [3, 1, 4, 1, 5, 2]
    g, wt = wgraph(7, [(i, i + 1, w[i]) for i in range(6)])
    pref = np.concatenate([[0], np.cumsum(w)])
    ident = np.arange(7, dtype=np.int32)
    # identity order: every h <= v outranks the whole h..v path
    assert rows(O.pll_weighted(g.off, g.col, wt, ident)) == [[(h, int(pref[v] - pref[h])) for h in range(v + 1)]
                                                              for v in range(7)]
    # reversed order (rank r = vertex 6 - r): hubs are the vertices h >= v
    rev = ident[::-1].copy()
    assert rows(O.pll_weighted(g.off, g.col, wt, rev)) == [
        sorted((6 - h, int(pref[h] - pref[v])) for h in range(v, 7)) for v in range(7)]


@pytest.mark.parametrize("w02,want2", [
    (5, [(0, 1), (2, 0)]),          # 0-1-2 (length 2) is the only shortest path: vertex 1 (rank 0) is on it
    (2, [(0, 1), (2, 0)]),          # tie: 0-2 and 0-1-2 are both shortest; P_02 still holds vertex 1
    (1, [(0, 1), (1, 1), (2, 0)]),  # the direct edge is strictly shorter: vertex 0 (rank 1) is a hub of 2
])
def test_triangle_by_hand(w02, want2):
    """Triangle 0-1 (1), 1-2 (1), 0-2 (w02) under order [1, 0, 2] (vertex 1
    has rank 0, vertex 0 rank 1, vertex 2 rank 2)."""
    g, wt = wgraph(3, [(0, 1, 1), (1, 2, 1), (0, 2, w02)])
    L = rows(O.pll_weighted(g.off, g.col, wt, np.array([1, 0, 2], np.int32)))
    assert L[1] == [(0, 0)]
    assert L[0] == [(0, 1), (1, 0)]
    assert L[2] == want2


def test_weighted_invariants_on_chung_lu():
    g = G.chung_lu_graph(3000, 8.0, 2.1, 6)
    wt = G.edge_weights(g, 1, 7, 2)
    order = G.degree_order(g)
    L = O.pll_weighted(g.off, g.col, wt, order)
    rank = np.empty(g.n, dtype=np.int64)
    rank[order] = np.arange(g.n)
    a = sp.csr_matrix((wt.astype(np.float64), g.col, g.off), shape=(g.n, g.n))
    rng = np.random.default_rng(3)
    for v in rng.choice(g.n, 30, replace=False):
        D = shortest_path(a, method="D", directed=True, indices=int(v))
        h, d = L.row(int(v))
        assert np.all(np.diff(h.astype(np.int64)) > 0)
        assert h[-1] == rank[v] and d[-1] == 0
        assert np.array_equal(d.astype(np.float64), D[order[h]])
        hh, dd = O.chhl_row_weighted(g.off, g.col, wt, order, int(v))
        assert np.array_equal(hh, h) and np.array_equal(dd, d)


def test_edge_weights_generator():
    g = G.rmat_graph(9, 8, 2)
    wt = G.edge_weights(g, 1, 7, 11)
    assert wt.min() >= 1 and wt.max() <= 7 and len(np.unique(wt)) == 7
    src = np.repeat(np.arange(g.n), np.diff(g.off))
    back = {(int(u), int(v)): int(w) for u, v, w in zip(src, g.col, wt)}
    assert all(back[(v, u)] == w for (u, v), w in back.items())      # both arcs of an edge alike
    assert np.array_equal(wt, G.edge_weights(g, 1, 7, 11))           # seeded
    assert not np.array_equal(wt, G.edge_weights(g, 1, 7, 12))


def test_weighted_distance_overflow_is_reported():
    """Label distances are uint8 up to 254: a path whose weighted length
    passes 254 makes the oracle refuse (the GPU build reports
    PLB_ERR_DIST_OVERFLOW for the same input), one just below does not."""
    g, wt = wgraph(4, [(0, 1, 100), (1, 2, 100), (2, 3, 54)])
    L = O.pll_weighted(g.off, g.col, wt, np.arange(4, dtype=np.int32))
    assert L.max_dist == 254 and rows(L)[3] == [(0, 254), (1, 154), (2, 54), (3, 0)]
    g, wt = wgraph(4, [(0, 1, 100), (1, 2, 100), (2, 3, 55)])
    with pytest.raises(OverflowError):
        O.pll_weighted(g.off, g.col, wt, np.arange(4, dtype=np.int32))


def test_constant_weight_generator_and_labels():
    g = G.rmat_graph(8, 4, 5)
    wt = G.edge_weights(g, 3, 3, 1)
    assert np.all(wt == 3)
    order = G.degree_order(g)
    W = O.pll_weighted(g.off, g.col, wt, order)
    U = O.pll(g.off, g.col, order)
    assert np.array_equal(W.hub, U.hub) and np.array_equal(W.dist.astype(np.int32), 3 * U.dist.astype(np.int32))
    with pytest.raises(ValueError):
        G.edge_weights(g, 0, 3, 1)
