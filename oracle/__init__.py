"""CPU oracle for canonical 2-hop distance labeling -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The GPU library never calls it and shares
no code with it.

Functions (each restates one definition or algorithm of the paper, Jin et al.,
"Pruned Landmark Labeling Meets Vertex Centric Computation"):

* ``pll``       Alg. 1, sequential pruned BFS per root in rank order (Sec. 2.1.1)
* ``vcpll``     Alg. 3, vertex-centric rounds with unique messages (Sec. 3.1)
* ``bvcpll``    Alg. 4 (BVC-PLL, Sec. 4.2): hubs in rank batches, a candidate
                bit-vector per vertex and batch, vertex-centric rounds
* ``chhl``      Def. 2, canonical labels by definition (one BFS per vertex)
* ``chhl_row``  Def. 2 for a single vertex (usable on large graphs)
* ``query``     2-hop distance query (Sec. 2.1)
* ``bfs``       textbook BFS distances
* ``pll_directed``  the directed form (Sec. 5.1): (L_in, L_out) by a forward
                and a backward pruned BFS per root
* ``chhl_directed`` Def. 2 for directed graphs: L_in(v) from the BFS over
                in-arcs, L_out(v) over out-arcs (``chhl`` on each CSR)
* ``query_directed`` d(s->t) from L_out(s) and L_in(t)
* ``pll_weighted``  weighted graphs (Sec. 5.1; the Sec. 6.4 baseline): Alg. 1
                with a pruned Dijkstra search per root
* ``chhl_weighted``, ``chhl_row_weighted``  Def. 2 for weighted graphs (one
                Dijkstra per vertex, best rank along the shortest-path DAG)
* ``dijkstra``  textbook Dijkstra distances

Labels come back as ``Labels(off, hub, dist)``: rows indexed by original id,
hub = rank (uint32), dist uint8, each row sorted by hub rank.  ``pll`` and
``vcpll`` also count, per vertex, the positive distance-check cost of Sec. 4.3
(``Labels.cost``: over the labels accepted at v, the other labels of v that
each check reads).

Pinning: ``tests/test_oracle.py`` (scipy all-pairs distances and the
shortest-path-set form of Def. 2, closed forms, invariants, paper identities),
``tests/test_oracle_directed.py``, ``tests/test_oracle_weighted.py``,
``tests/test_oracle_cost.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "libplboracle.so")
_lib = None


def build(verbose: bool = False) -> str:
    """Compile ``plb_oracle.c`` (gcc, host code)."""
    src = os.path.join(_HERE, "plb_oracle.c")
    tmp = _LIB_PATH + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-fPIC", "-shared", "-o", tmp, src]
    if verbose:
        print(" ".join(cmd))
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_LIB_PATH):
        build()
    lib = ctypes.CDLL(_LIB_PATH)
    P = ctypes.c_void_p
    I64 = ctypes.c_int64
    for name in ("oracle_pll", "oracle_vcpll", "oracle_chhl"):
        f = getattr(lib, name)
        f.argtypes = [I64, P, P, P]
        f.restype = P
    lib.oracle_pll_budget.argtypes = [I64, P, P, P, ctypes.c_double, ctypes.POINTER(ctypes.c_int64)]
    lib.oracle_pll_budget.restype = P
    lib.oracle_chhl_row.argtypes = [I64, P, P, P, ctypes.c_int32, P, P, I64]
    lib.oracle_chhl_row.restype = I64
    lib.oracle_labels_free.argtypes = [P]
    lib.oracle_labels_free.restype = None
    lib.oracle_labels_total.argtypes = [P]
    lib.oracle_labels_total.restype = I64
    lib.oracle_labels_max_dist.argtypes = [P]
    lib.oracle_labels_max_dist.restype = ctypes.c_int32
    lib.oracle_labels_rounds.argtypes = [P]
    lib.oracle_labels_rounds.restype = ctypes.c_int32
    lib.oracle_labels_stats.argtypes = [P]
    lib.oracle_labels_stats.restype = ctypes.POINTER(ctypes.c_int64)
    lib.oracle_labels_export.argtypes = [P, P, P, P]
    lib.oracle_labels_export.restype = None
    lib.oracle_labels_cost.argtypes = [P, P]
    lib.oracle_labels_cost.restype = None
    lib.oracle_labels_checks.argtypes = [P]
    lib.oracle_labels_checks.restype = I64
    lib.oracle_bvcpll.argtypes = [I64, P, P, P, I64]
    lib.oracle_bvcpll.restype = P
    lib.oracle_query.argtypes = [I64, P, P, P, P, P]
    lib.oracle_query.restype = None
    lib.oracle_bfs.argtypes = [I64, P, P, ctypes.c_int32, P]
    lib.oracle_bfs.restype = None
    lib.oracle_pll_directed.argtypes = [I64, P, P, P, P, P, ctypes.POINTER(ctypes.c_void_p)]
    lib.oracle_pll_directed.restype = P
    lib.oracle_query2.argtypes = [I64, P, P, P, P, P, P, P, P]
    lib.oracle_query2.restype = None
    for name in ("oracle_pll_weighted", "oracle_chhl_weighted"):
        f = getattr(lib, name)
        f.argtypes = [I64, P, P, P, P]
        f.restype = P
    lib.oracle_pll_weighted_budget.argtypes = [I64, P, P, P, P, ctypes.c_double, ctypes.POINTER(ctypes.c_int64)]
    lib.oracle_pll_weighted_budget.restype = P
    lib.oracle_chhl_row_weighted.argtypes = [I64, P, P, P, P, ctypes.c_int32, P, P, I64]
    lib.oracle_chhl_row_weighted.restype = I64
    lib.oracle_dijkstra.argtypes = [I64, P, P, P, ctypes.c_int32, P]
    lib.oracle_dijkstra.restype = None
    _lib = lib
    return lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


@dataclass
class Labels:
    off: np.ndarray   # int64[n+1]
    hub: np.ndarray   # uint32[total], hub RANK
    dist: np.ndarray  # uint8[total]
    max_dist: int = 0
    rounds: int = 0
    round_stats: np.ndarray | None = None  # VC-PLL: [round, (messages, unique, accepted, checks)]
    cost: np.ndarray | None = None  # PLL / VC-PLL: per vertex, positive distance-check cost (Sec. 4.3)
    checks: int = 0  # PLL: vertices reached over all pruned searches; BVC-PLL: messages sent

    @property
    def n(self) -> int:
        return int(self.off.shape[0] - 1)

    @property
    def total(self) -> int:
        return int(self.hub.shape[0])

    def row(self, v: int):
        a, b = int(self.off[v]), int(self.off[v + 1])
        return self.hub[a:b], self.dist[a:b]


def _csr_args(off, col, order):
    off = np.ascontiguousarray(off, dtype=np.int64)
    col = np.ascontiguousarray(col, dtype=np.int32)
    order = np.ascontiguousarray(order, dtype=np.int32)
    n = int(off.shape[0] - 1)
    if order.shape[0] != n:
        raise ValueError("order must have n entries")
    if col.shape[0] == 0:
        col = np.zeros(1, dtype=np.int32)
    return n, off, col, order


def _export(h, n) -> Labels:
    lib = _load()
    total = lib.oracle_labels_total(h)
    off = np.zeros(n + 1, dtype=np.int64)
    hub = np.empty(max(total, 1), dtype=np.uint32)
    dist = np.empty(max(total, 1), dtype=np.uint8)
    lib.oracle_labels_export(h, _p(off), _p(hub), _p(dist))
    rounds = lib.oracle_labels_rounds(h)
    st = lib.oracle_labels_stats(h)
    stats = np.ctypeslib.as_array(st, shape=(256, 4)).copy() if rounds else None
    cost = np.zeros(max(n, 1), dtype=np.int64)
    lib.oracle_labels_cost(h, _p(cost))
    lab = Labels(off, hub[:total].copy(), dist[:total].copy(), lib.oracle_labels_max_dist(h),
                 rounds, stats, cost[:n], int(lib.oracle_labels_checks(h)))
    lib.oracle_labels_free(h)
    return lab


def _run(fname, off, col, order) -> Labels:
    n, off, col, order = _csr_args(off, col, order)
    h = getattr(_load(), fname)(n, _p(off), _p(col), _p(order))
    if not h:
        raise OverflowError("label distance above 254 (or out of memory)")
    return _export(h, n)


def pll(off, col, order) -> Labels:
    """Alg. 1 (PLL with the small revision)."""
    return _run("oracle_pll", off, col, order)


def pll_budget(off, col, order, seconds: float):
    """Alg. 1 over the roots in rank order, stopped once ``seconds`` have
    elapsed (checked between roots).  Returns (labels so far, roots done,
    elapsed seconds); a bounded sample for timing the oracle."""
    import time

    n, off, col, order = _csr_args(off, col, order)
    done = ctypes.c_int64(0)
    t0 = time.perf_counter()
    h = _load().oracle_pll_budget(n, _p(off), _p(col), _p(order), float(seconds), ctypes.byref(done))
    el = time.perf_counter() - t0
    if not h:
        raise OverflowError("label distance above 254 (or out of memory)")
    return _export(h, n), int(done.value), el


def vcpll(off, col, order) -> Labels:
    """Alg. 3 (VC-PLL), with per-round message / unique / accepted / check counts."""
    return _run("oracle_vcpll", off, col, order)


def bvcpll(off, col, order, batch: int) -> Labels:
    """Alg. 4 (BVC-PLL) with hub batches of ``batch`` consecutive ranks;
    ``checks`` counts the messages sent (one distance check each)."""
    n, off, col, order = _csr_args(off, col, order)
    h = _load().oracle_bvcpll(n, _p(off), _p(col), _p(order), int(batch))
    if not h:
        raise OverflowError("label distance above 254 (or out of memory)")
    return _export(h, n)


def chhl(off, col, order) -> Labels:
    """Def. 2 by definition for every vertex (O(n m); small graphs)."""
    return _run("oracle_chhl", off, col, order)


def chhl_row(off, col, order, v: int):
    """Def. 2 for one vertex v: (hub ranks, distances), sorted by rank."""
    n, off, col, order = _csr_args(off, col, order)
    hub = np.empty(max(n, 1), dtype=np.uint32)
    dist = np.empty(max(n, 1), dtype=np.uint8)
    k = _load().oracle_chhl_row(n, _p(off), _p(col), _p(order), int(v), _p(hub), _p(dist), n)
    return hub[:k].copy(), dist[:k].copy()


def query(labels: Labels, pairs) -> np.ndarray:
    """2-hop query for int32 pairs [q, 2]; -1 where no hub is common."""
    pairs = np.ascontiguousarray(pairs, dtype=np.int32).reshape(-1, 2)
    q = int(pairs.shape[0])
    out = np.empty(max(q, 1), dtype=np.int32)
    hub = labels.hub if labels.total else np.zeros(1, np.uint32)
    dist = labels.dist if labels.total else np.zeros(1, np.uint8)
    if q:
        _load().oracle_query(q, _p(labels.off), _p(hub), _p(dist), _p(pairs), _p(out))
    return out[:q]


def pll_directed(off_out, col_out, off_in, col_in, order):
    """Directed PLL (Sec. 5.1): returns (L_in, L_out); rows by original id,
    hubs as ranks.  off_in/col_in is the transpose of off_out/col_out."""
    n, off_out, col_out, order = _csr_args(off_out, col_out, order)
    _, off_in, col_in, _ = _csr_args(off_in, col_in, order)
    lout = ctypes.c_void_p()
    h = _load().oracle_pll_directed(n, _p(off_out), _p(col_out), _p(off_in), _p(col_in), _p(order),
                                    ctypes.byref(lout))
    if not h:
        raise OverflowError("label distance above 254 (or out of memory)")
    return _export(h, n), _export(lout.value, n)


def chhl_directed(off_out, col_out, off_in, col_in, order):
    """Def. 2 for directed graphs: (L_in, L_out).  h is in L_in(v) iff it
    outranks every vertex of every shortest h->v path: the per-vertex BFS of
    ``chhl`` over the in-arcs; L_out likewise over the out-arcs."""
    return chhl(off_in, col_in, order), chhl(off_out, col_out, order)


def query_directed(lout: Labels, lin: Labels, pairs) -> np.ndarray:
    """d(s->t) for int32 pairs [q, 2] from L_out(s) and L_in(t); -1 if none."""
    pairs = np.ascontiguousarray(pairs, dtype=np.int32).reshape(-1, 2)
    q = int(pairs.shape[0])
    out = np.empty(max(q, 1), dtype=np.int32)

    def arrs(L):
        return (L.off, L.hub if L.total else np.zeros(1, np.uint32), L.dist if L.total else np.zeros(1, np.uint8))

    if q:
        a, b = arrs(lout), arrs(lin)
        _load().oracle_query2(q, _p(a[0]), _p(a[1]), _p(a[2]), _p(b[0]), _p(b[1]), _p(b[2]), _p(pairs), _p(out))
    return out[:q]


def bfs(off, col, src: int) -> np.ndarray:
    off = np.ascontiguousarray(off, dtype=np.int64)
    col = np.ascontiguousarray(col, dtype=np.int32)
    n = int(off.shape[0] - 1)
    dist = np.empty(max(n, 1), dtype=np.int32)
    if col.shape[0] == 0:
        col = np.zeros(1, dtype=np.int32)
    _load().oracle_bfs(n, _p(off), _p(col), int(src), _p(dist))
    return dist[:n]


def _weights(wt, nnz: int) -> np.ndarray:
    wt = np.ascontiguousarray(wt, dtype=np.uint8)
    if wt.shape[0] != nnz:
        raise ValueError("one weight per arc")
    return wt if nnz else np.ones(1, dtype=np.uint8)


def pll_weighted(off, col, wt, order) -> Labels:
    """Alg. 1 on a weighted graph: one pruned Dijkstra search per root in
    rank order (the PLL baseline of Sec. 6.4).  ``wt`` holds one uint8
    weight >= 1 per arc, equal in both directions."""
    nnz = int(np.asarray(col).shape[0])
    n, off, col, order = _csr_args(off, col, order)
    wt = _weights(wt, nnz)
    h = _load().oracle_pll_weighted(n, _p(off), _p(col), _p(wt), _p(order))
    if not h:
        raise OverflowError("label distance above 254 (or out of memory)")
    return _export(h, n)


def pll_weighted_budget(off, col, wt, order, seconds: float):
    """``pll_weighted`` stopped once ``seconds`` have elapsed (between roots):
    (labels so far, roots done, elapsed seconds)."""
    import time

    nnz = int(np.asarray(col).shape[0])
    n, off, col, order = _csr_args(off, col, order)
    wt = _weights(wt, nnz)
    done = ctypes.c_int64(0)
    t0 = time.perf_counter()
    h = _load().oracle_pll_weighted_budget(n, _p(off), _p(col), _p(wt), _p(order), float(seconds),
                                           ctypes.byref(done))
    el = time.perf_counter() - t0
    if not h:
        raise OverflowError("label distance above 254 (or out of memory)")
    return _export(h, n), int(done.value), el


def chhl_weighted(off, col, wt, order) -> Labels:
    """Def. 2 on a weighted graph for every vertex (n Dijkstra runs)."""
    nnz = int(np.asarray(col).shape[0])
    n, off, col, order = _csr_args(off, col, order)
    wt = _weights(wt, nnz)
    h = _load().oracle_chhl_weighted(n, _p(off), _p(col), _p(wt), _p(order))
    return _export(h, n)


def chhl_row_weighted(off, col, wt, order, v: int):
    """Def. 2 on a weighted graph for one vertex: (hub ranks, distances)."""
    nnz = int(np.asarray(col).shape[0])
    n, off, col, order = _csr_args(off, col, order)
    wt = _weights(wt, nnz)
    hub = np.empty(max(n, 1), dtype=np.uint32)
    dist = np.empty(max(n, 1), dtype=np.uint8)
    k = _load().oracle_chhl_row_weighted(n, _p(off), _p(col), _p(wt), _p(order), int(v), _p(hub), _p(dist), n)
    return hub[:k].copy(), dist[:k].copy()


def dijkstra(off, col, wt, src: int) -> np.ndarray:
    """Textbook Dijkstra distances from src (-1 unreachable)."""
    nnz = int(np.asarray(col).shape[0])
    off = np.ascontiguousarray(off, dtype=np.int64)
    col = np.ascontiguousarray(col, dtype=np.int32)
    n = int(off.shape[0] - 1)
    wt = _weights(wt, nnz)
    if col.shape[0] == 0:
        col = np.zeros(1, dtype=np.int32)
    dist = np.empty(max(n, 1), dtype=np.int32)
    _load().oracle_dijkstra(n, _p(off), _p(col), _p(wt), int(src), _p(dist))
    return dist[:n]
