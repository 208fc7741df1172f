"""Pins for the CPU oracle (no GPU).

The oracle is checked against things other than itself:

* Def. 2 restated from scratch: all-pairs distances from scipy's
  ``shortest_path`` (a library routine), the shortest-path vertex set
  P_uv = {w : d(u,w) + d(w,v) = d(u,v)}, and "h is a hub of v iff h has the
  highest rank in P_hv".  This shares nothing with the oracle's BFS-DAG form.
* hand-derived golden labels (tests/golden/*.txt, Def. 2);
* closed forms: star, complete graph, path;
* the query formula (Sec. 2.1) against scipy all-pairs distances;
* invariants: hierarchy (hub outranks owner), (v,0) in L(v), hub-sorted rows,
  exact stored distances (Cor. 1), disconnected parts never share hubs;
* Thm. 1 / Sec. 4.2: PLL, VC-PLL and the definition give identical labels;
* Lemma 1: every label arrives at distance d(u,v) (VC-PLL rounds);
* distance overflow (uint8 labels) is reported.
"""
import os

import numpy as np
import pytest
import scipy.sparse as sp
from scipy.sparse.csgraph import shortest_path

import oracle as O
from paper_1906_12018_gb300 import graphs as G

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ----------------------------------------------------------------- helpers
def apsp(g):
    n = g.n
    if n == 0:
        return np.zeros((0, 0))
    a = sp.csr_matrix((np.ones(g.nnz), g.col, g.off), shape=(n, n))
    return shortest_path(a, method="D", unweighted=True, directed=False)


def labels_by_definition(g, order):
    """Def. 2 from all-pairs distances: h in L(v) iff rank(h) = min rank over P_hv."""
    n = g.n
    D = apsp(g)
    rank = np.empty(n, dtype=np.int64)
    rank[order] = np.arange(n)
    rows = []
    for v in range(n):
        row = []
        for h in range(n):
            if not np.isfinite(D[h, v]):
                continue
            on_path = np.isfinite(D[h]) & (D[h] + D[:, v] == D[h, v])
            if rank[on_path].min() == rank[h]:
                row.append((int(rank[h]), int(D[h, v])))
        rows.append(sorted(row))
    return rows


def rows_of(lab):
    return [list(zip(lab.row(v)[0].tolist(), lab.row(v)[1].tolist())) for v in range(lab.n)]


def random_graph(rng, n, p):
    iu = np.triu_indices(n, 1)
    keep = rng.random(iu[0].shape[0]) < p
    return G.from_edges(n, zip(iu[0][keep], iu[1][keep]))


def tiny_graphs():
    rng = np.random.default_rng(7)
    out = []
    for n, p in [(1, 0.0), (2, 1.0), (5, 0.5), (8, 0.3), (12, 0.25), (16, 0.15), (20, 0.1), (24, 0.3)]:
        out.append((f"er{n}-{p}", random_graph(rng, n, p)))
    # tree, grid, cycle, disconnected union, star, complete
    par = [rng.integers(0, i) for i in range(1, 20)]
    out.append(("tree20", G.from_edges(20, [(i + 1, par[i]) for i in range(19)])))
    grid = [(r * 5 + c, r * 5 + c + 1) for r in range(4) for c in range(4)]
    grid += [(r * 5 + c, (r + 1) * 5 + c) for r in range(3) for c in range(5)]
    out.append(("grid4x5", G.from_edges(20, grid)))
    out.append(("cycle9", G.from_edges(9, [(i, (i + 1) % 9) for i in range(9)])))
    out.append(("two-parts", G.from_edges(10, [(0, 1), (1, 2), (2, 0), (5, 6), (6, 7), (7, 8), (8, 5), (5, 7)])))
    out.append(("star7", G.from_edges(7, [(0, i) for i in range(1, 7)])))
    out.append(("K6", G.from_edges(6, [(i, j) for i in range(6) for j in range(i + 1, 6)])))
    return out


def orders_for(g, rng):
    yield G.degree_order(g)
    yield np.arange(g.n, dtype=np.int32)
    yield rng.permutation(g.n).astype(np.int32)


# ------------------------------------------------------- Def. 2 (pinned)
@pytest.mark.parametrize("name,g", tiny_graphs(), ids=lambda x: x if isinstance(x, str) else "")
def test_definition_matches_shortest_path_sets(name, g):
    rng = np.random.default_rng(11)
    for order in orders_for(g, rng):
        want = labels_by_definition(g, order)
        assert rows_of(O.chhl(g.off, g.col, order)) == want
        assert rows_of(O.pll(g.off, g.col, order)) == want
        assert rows_of(O.vcpll(g.off, g.col, order)) == want


def load_golden(fname):
    n, edges, order, rows = 0, [], None, {}
    with open(os.path.join(GOLDEN, fname)) as f:
        for line in f:
            t = line.split()
            if not t or t[0].startswith("#"):
                continue
            if t[0] == "n":
                n = int(t[1])
            elif t[0] == "e":
                edges.append((int(t[1]), int(t[2])))
            elif t[0] == "o":
                order = np.array([int(x) for x in t[1:]], dtype=np.int32)
            elif t[0] == "L":
                rows[int(t[1])] = [tuple(int(y) for y in x.split(":")) for x in t[2:]]
    if order is None:
        order = np.arange(n, dtype=np.int32)
    return G.from_edges(n, edges), order, [rows[v] for v in range(n)]


@pytest.mark.parametrize("fname", ["cycle4.txt", "paw.txt"])
def test_golden_hand_derived(fname):
    g, order, want = load_golden(fname)
    assert labels_by_definition(g, order) == want
    for f in (O.pll, O.vcpll, O.chhl):
        assert rows_of(f(g.off, g.col, order)) == want


# ------------------------------------------------------------ closed forms
def test_star_closed_form():
    n = 50
    g = G.from_edges(n, [(0, i) for i in range(1, n)])
    order = G.degree_order(g)
    assert order[0] == 0
    lab = O.pll(g.off, g.col, order)
    assert lab.total == 2 * n - 1
    for v in range(1, n):
        h, d = lab.row(v)
        assert h.tolist() == [0, int(np.where(order == v)[0][0])] and d.tolist() == [1, 0]


def test_complete_graph_closed_form():
    n = 30
    g = G.from_edges(n, [(i, j) for i in range(n) for j in range(i + 1, n)])
    order = np.arange(n, dtype=np.int32)
    lab = O.pll(g.off, g.col, order)
    assert lab.total == n * (n + 1) // 2
    for i in range(n):
        h, d = lab.row(i)
        assert h.tolist() == list(range(i + 1))
        assert d.tolist() == [1] * i + [0]


def test_path_closed_form():
    # path 0-1-...-(n-1), rank = position: every j <= i is a hub of i at i-j
    n = 40
    g = G.from_edges(n, [(i, i + 1) for i in range(n - 1)])
    order = np.arange(n, dtype=np.int32)
    lab = O.vcpll(g.off, g.col, order)
    assert lab.total == n * (n + 1) // 2
    assert lab.rounds == n  # the last round accepts nothing
    for i in range(n):
        h, d = lab.row(i)
        assert h.tolist() == list(range(i + 1))
        assert d.tolist() == [i - j for j in range(i + 1)]


def test_isolated_and_empty():
    g = G.from_edges(5, [(0, 1)])
    order = G.degree_order(g)
    lab = O.pll(g.off, g.col, order)
    assert lab.total == 1 + 2 + 1 + 1 + 1
    for v in (2, 3, 4):
        assert lab.row(v)[1].tolist() == [0]
    q = O.query(lab, [[0, 1], [0, 2], [3, 3], [2, 4]])
    assert q.tolist() == [1, -1, 0, -1]
    g0 = G.from_edges(0, [])
    assert O.pll(g0.off, g0.col, np.zeros(0, np.int32)).total == 0


def test_distance_overflow_reported():
    n = 300  # a path has distances up to 299 > 254
    g = G.from_edges(n, [(i, i + 1) for i in range(n - 1)])
    with pytest.raises(OverflowError):
        O.pll(g.off, g.col, np.arange(n, dtype=np.int32))
    with pytest.raises(OverflowError):
        O.vcpll(g.off, g.col, np.arange(n, dtype=np.int32))
    # 255 vertices: the largest distance is exactly 254
    g = G.from_edges(255, [(i, i + 1) for i in range(254)])
    assert O.pll(g.off, g.col, np.arange(255, dtype=np.int32)).max_dist == 254


# -------------------------------------------------------------- the query
@pytest.mark.parametrize("name,g", tiny_graphs()[2:], ids=lambda x: x if isinstance(x, str) else "")
def test_query_equals_apsp(name, g):
    order = G.degree_order(g)
    lab = O.pll(g.off, g.col, order)
    D = apsp(g)
    s, t = np.meshgrid(np.arange(g.n), np.arange(g.n), indexing="ij")
    pairs = np.stack([s.ravel(), t.ravel()], 1)
    got = O.query(lab, pairs)
    want = np.where(np.isfinite(D.ravel()), D.ravel(), -1).astype(np.int64)
    assert np.array_equal(got, want)


@pytest.mark.parametrize("name,g", tiny_graphs(), ids=lambda x: x if isinstance(x, str) else "")
def test_bfs_equals_apsp(name, g):
    """The textbook BFS that checks sampled GPU queries on the large
    workloads, pinned to scipy's all-pairs distances from every source."""
    D = apsp(g)
    for s in range(g.n):
        want = np.where(np.isfinite(D[s]), D[s], -1).astype(np.int64)
        assert np.array_equal(O.bfs(g.off, g.col, s), want), (name, s)


def test_bfs_equals_scipy_on_rmat12():
    g = G.workload("rmat12")
    a = sp.csr_matrix((np.ones(g.nnz), g.col, g.off), shape=(g.n, g.n))
    src = [0, 1, 17, g.n // 2, g.n - 1]
    D = shortest_path(a, method="D", unweighted=True, directed=False, indices=src)
    for i, s in enumerate(src):
        want = np.where(np.isfinite(D[i]), D[i], -1).astype(np.int64)
        assert np.array_equal(O.bfs(g.off, g.col, s), want), s


# ----------------------------------------------------- R-MAT 2^12 workload
@pytest.fixture(scope="module")
def rmat12():
    g = G.workload("rmat12")
    return g, G.degree_order(g)


def test_rmat12_three_forms_agree(rmat12):
    g, order = rmat12
    a = O.pll(g.off, g.col, order)
    b = O.vcpll(g.off, g.col, order)
    c = O.chhl(g.off, g.col, order)
    for x in (b, c):
        assert np.array_equal(a.off, x.off)
        assert np.array_equal(a.hub, x.hub)
        assert np.array_equal(a.dist, x.dist)


def test_rmat12_invariants_and_queries(rmat12):
    g, order = rmat12
    lab = O.pll(g.off, g.col, order)
    n = g.n
    rank = np.empty(n, dtype=np.int64)
    rank[order] = np.arange(n)
    D = apsp(g)
    for v in range(n):
        h, d = lab.row(v)
        assert np.all(np.diff(h.astype(np.int64)) > 0)       # sorted, no duplicates
        assert h[-1] == rank[v] and d[-1] == 0               # (v,0) is the last entry
        assert np.all(h.astype(np.int64) <= rank[v])         # hierarchy
        assert np.array_equal(d.astype(np.int64), D[order[h.astype(np.int64)], v].astype(np.int64))  # exact
    pairs = G.uniform_pairs(n, 10_000, 1)
    got = O.query(lab, pairs)
    want = D[pairs[:, 0], pairs[:, 1]]
    assert np.array_equal(got, np.where(np.isfinite(want), want, -1).astype(np.int64))


def test_vcpll_round_structure(rmat12):
    """Round d accepts only labels at distance d (Cor. 1); rounds stop one
    round after the largest distance; every accepted label was a unique
    message and every unique message was checked at least once."""
    g, order = rmat12
    lab = O.vcpll(g.off, g.col, order)
    assert lab.rounds == lab.max_dist + 1
    st = lab.round_stats
    acc = st[1:lab.rounds + 1, 2]
    counts = np.bincount(lab.dist, minlength=lab.rounds + 1)
    assert np.array_equal(acc, counts[1:lab.rounds + 1])
    assert np.all(st[:, 1] <= st[:, 0])        # unique <= messages
    assert np.all(st[:, 2] <= st[:, 1])        # accepted <= unique
    assert st[1, 0] == g.m                     # round 1: one message per edge, to the lower-ranked end


def test_disconnected_union_has_no_cross_hubs():
    a = G.rmat_graph(8, 4, 5)
    b = G.rmat_graph(8, 4, 6)
    off = np.concatenate([a.off, b.off[1:] + a.off[-1]])
    col = np.concatenate([a.col, b.col + a.n])
    order = np.concatenate([G.degree_order(a), G.degree_order(b) + a.n]).astype(np.int32)
    lab = O.pll(off, col, order)
    la = O.pll(a.off, a.col, G.degree_order(a))
    lb = O.pll(b.off, b.col, G.degree_order(b))
    assert lab.total == la.total + lb.total
    assert np.array_equal(lab.hub[: la.total], la.hub)
    assert np.array_equal(lab.hub[la.total:], lb.hub + a.n)


def test_chhl_row_matches_full(rmat12):
    g, order = rmat12
    full = O.pll(g.off, g.col, order)
    for v in [0, 1, 17, g.n // 2, g.n - 1]:
        h, d = O.chhl_row(g.off, g.col, order, v)
        fh, fd = full.row(v)
        assert np.array_equal(h, fh) and np.array_equal(d, fd)


@pytest.mark.parametrize("i", [12, 18, 19, 25])
def test_batch_workload_graphs_match_definition(i):
    """Graphs of the batched workload (even i: R-MAT + LCC; odd i: Chung-Lu
    with isolated vertices): Alg. 1 and Alg. 3 equal Def. 2 computed by
    brute force, one BFS per vertex."""
    g = G.small_graph(i)
    order = G.degree_order(g)
    ref = O.chhl(g.off, g.col, order)
    for L in (O.pll(g.off, g.col, order), O.vcpll(g.off, g.col, order)):
        assert np.array_equal(L.off, ref.off) and np.array_equal(L.hub, ref.hub) and np.array_equal(L.dist, ref.dist)
