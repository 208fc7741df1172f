"""The round structure of the weighted build (rounds by distance value, Sec.
5.1's weighted graphs read with Alg. 3's snapshot check), modeled in plain
Python on small graphs, gives exactly the canonical labels of Def. 2 (the
oracle's Dijkstra form) -- no recheck pass needed.  The model shares nothing
with the GPU code; it pins the reading the GPU build relies on."""
import numpy as np
import pytest

import oracle as O
from paper_1906_12018_gb300 import graphs as G


def distance_rounds(n, adj, rank):
    """adj[v] = [(a, w)]; round d accepts labels at distance d: v gathers the
    hubs h (rank(h) < rank(v)) of the round-(d - w) frontiers of its
    neighbours a (w = w(a, v)), skips hubs it has, and accepts h unless a hub
    x of both has d(h, x) + d(x, v) <= d in the labels of rounds < d."""
    L = [{v: 0} for v in range(n)]
    front = {0: [{v} for v in range(n)]}
    maxw = max([w for row in adj for _, w in row] or [1])
    d, last = 0, 0
    while d - last < maxw:
        d += 1
        new = []
        for v in range(n):
            cand = set()
            for a, w in adj[v]:
                if d - w >= 0:
                    cand |= {h for h in front[d - w][a] if rank[h] < rank[v]}
            acc = set()
            for h in cand - set(L[v]):
                if not any(x in L[h] and L[h][x] + dv <= d for x, dv in L[v].items()):
                    acc.add(h)
            new.append(acc)
        for v in range(n):
            for h in new[v]:
                L[v][h] = d
        front[d] = new
        if any(new):
            last = d
    return L


def random_weighted(n, p, wmax, rng):
    m = np.triu(rng.random((n, n)) < p, 1)
    s, t = np.nonzero(m)
    w = rng.integers(1, wmax + 1, size=len(s))
    g = G.clean_csr(n, np.concatenate([s, t]), np.concatenate([t, s]))
    key = {(int(a), int(b)): int(x) for a, b, x in zip(s, t, w)}
    src = np.repeat(np.arange(n), np.diff(g.off))
    wt = np.array([key[(min(a, b), max(a, b))] for a, b in zip(src, g.col)], dtype=np.uint8)
    adj = [[(int(g.col[j]), int(wt[j])) for j in range(g.off[v], g.off[v + 1])] for v in range(n)]
    return g, wt, adj


@pytest.mark.parametrize("seed", range(12))
def test_distance_rounds_give_def2(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(5, 28))
    g, wt, adj = random_weighted(n, float(rng.uniform(0.1, 0.5)), int(rng.choice([2, 3, 7, 12])), rng)
    for order in (G.degree_order(g), rng.permutation(n).astype(np.int32)):
        rank = np.empty(n, dtype=np.int64)
        rank[order] = np.arange(n)
        L = distance_rounds(n, adj, rank)
        ref = O.chhl_weighted(g.off, g.col, wt, order)
        for v in range(n):
            h, dd = ref.row(v)
            got = sorted((int(rank[x]), dx) for x, dx in L[v].items())
            assert got == list(zip(h.tolist(), dd.tolist())), (seed, v)


def hop_rounds_without_recheck(n, adj, rank):
    """The direct form Sec. 5.1 warns about: rounds by hop count, candidate
    distance d(h, a) + w, the same snapshot check, labels never revised."""
    L = [{v: 0} for v in range(n)]
    front = [{v: 0} for v in range(n)]
    for _ in range(4 * n):
        new = []
        for v in range(n):
            best = {}
            for a, w in adj[v]:
                for h, dh in front[a].items():
                    if rank[h] < rank[v] and h not in L[v]:
                        best[h] = min(best.get(h, 1 << 30), dh + w)
            acc = {}
            for h, dd in best.items():
                if not any(x in L[h] and L[h][x] + dv <= dd for x, dv in L[v].items()):
                    acc[h] = dd
            new.append(acc)
        for v in range(n):
            L[v].update(new[v])
        front = new
        if not any(new):
            break
    return L


def test_hop_rounds_alone_are_not_canonical():
    """Triangle 0-1 (1), 1-2 (1), 0-2 (5), vertex 1 ranked last: by hops,
    vertex 2 first meets hub 0 over the direct edge at distance 5 and keeps
    it; the shortest 0-2 path (length 2) comes one round later, when 0 is
    already a hub of 2.  Rounds by distance accept (0, 2) instead."""
    adj = [[(1, 1), (2, 5)], [(0, 1), (2, 1)], [(0, 5), (1, 1)]]
    rank = np.array([0, 2, 1])
    hop = hop_rounds_without_recheck(3, adj, rank)
    dist = distance_rounds(3, adj, rank)
    assert hop[2][0] == 5          # a label at a distance that is not d(0, 2)
    assert dist[2][0] == 2         # the canonical entry
