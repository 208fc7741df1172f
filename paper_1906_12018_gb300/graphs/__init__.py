"""Seeded synthetic graph workloads (inputs only; none of the labeling arithmetic).

The C library ``libplbgen.so`` (built from ``gen.c``) does the heavy lifting;
this module marshals numpy arrays.  Every function is deterministic in its seed
and independent of the thread count.

Workloads (sizes of the paper's power-law graphs, Table 2, stand in for the
real datasets, which are not available here):

* ``rmat_graph``     R-MAT, (a,b,c,d) = (0.57,0.19,0.19,0.05), cleaned, optional LCC
* ``chung_lu_graph`` Chung-Lu, weights (i+1)^(-1/(gamma-1)), cleaned
* ``degree_order``   rank -> id, degree descending, ties by smaller id (Sec. 6.1)
* ``uniform_pairs``  i.i.d. uniform query pairs
* ``edge_weights``   seeded uniform integer weights per undirected edge (both arcs alike)
* ``workload``       the named labeling workloads used by tests and the benchmark
"""
from __future__ import annotations

import ctypes
import math
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "libplbgen.so")
_lib = None

RMAT_ABC = (0.57, 0.19, 0.19)


def build(verbose: bool = False) -> str:
    """Compile ``gen.c`` into ``libplbgen.so`` (host code, gcc)."""
    import subprocess

    src = os.path.join(_HERE, "gen.c")
    tmp = _LIB_PATH + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
           "-o", tmp, src, "-lm"]
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
    U64 = ctypes.c_uint64
    D = ctypes.c_double
    lib.gen_rmat_edges.argtypes = [ctypes.c_int, I64, D, D, D, U64, I64, P, P]
    lib.gen_rmat_edges.restype = ctypes.c_int
    lib.gen_chung_lu_edges.argtypes = [I64, I64, D, U64, P, P]
    lib.gen_chung_lu_edges.restype = ctypes.c_int
    lib.gen_clean_csr.argtypes = [I64, I64, P, P, P, P]
    lib.gen_clean_csr.restype = I64
    lib.gen_lcc_map.argtypes = [I64, P, P, P]
    lib.gen_lcc_map.restype = I64
    lib.gen_induce.argtypes = [I64, P, P, P, P, P]
    lib.gen_induce.restype = I64
    lib.gen_degree_order.argtypes = [I64, P, P]
    lib.gen_degree_order.restype = None
    lib.gen_uniform_pairs.argtypes = [I64, I64, U64, P]
    lib.gen_uniform_pairs.restype = None
    lib.gen_log_uniform_size.argtypes = [U64, D, D]
    lib.gen_log_uniform_size.restype = I64
    lib.gen_uniform_int.argtypes = [U64, U64, U64, I64, I64]
    lib.gen_uniform_int.restype = I64
    lib.gen_uniform01.argtypes = [U64, U64, U64]
    lib.gen_uniform01.restype = D
    lib.gen_draw.argtypes = [U64, U64, U64]
    lib.gen_draw.restype = U64
    _lib = lib
    return lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


@dataclass
class Graph:
    """Undirected simple graph as a symmetric CSR with ascending rows."""

    off: np.ndarray  # int64[n+1]
    col: np.ndarray  # int32[nnz]
    name: str = ""

    @property
    def n(self) -> int:
        return int(self.off.shape[0] - 1)

    @property
    def nnz(self) -> int:
        return int(self.col.shape[0])

    @property
    def m(self) -> int:
        """Undirected edges."""
        return self.nnz // 2

    def degrees(self) -> np.ndarray:
        return np.diff(self.off)


def clean_csr(n: int, src: np.ndarray, dst: np.ndarray) -> Graph:
    """Symmetrise, drop self-loops and duplicates; rows sorted ascending."""
    lib = _load()
    src = np.ascontiguousarray(src, dtype=np.int32)
    dst = np.ascontiguousarray(dst, dtype=np.int32)
    m = int(src.shape[0])
    off = np.zeros(n + 1, dtype=np.int64)
    col = np.empty(max(2 * m, 1), dtype=np.int32)
    nnz = lib.gen_clean_csr(n, m, _p(src), _p(dst), _p(off), _p(col))
    if nnz < 0:
        raise ValueError("edge endpoint out of range")
    return Graph(off, col[:nnz].copy())


def from_edges(n: int, edges) -> Graph:
    """Graph from an iterable of (u, v) pairs (test helper)."""
    e = np.asarray(list(edges), dtype=np.int64).reshape(-1, 2)
    return clean_csr(n, e[:, 0].astype(np.int32), e[:, 1].astype(np.int32))


def largest_component(g: Graph) -> Graph:
    lib = _load()
    new_id = np.empty(max(g.n, 1), dtype=np.int32)
    size = lib.gen_lcc_map(g.n, _p(g.off), _p(g.col), _p(new_id))
    off = np.zeros(size + 1, dtype=np.int64)
    col = np.empty(max(g.nnz, 1), dtype=np.int32)
    nnz = lib.gen_induce(g.n, _p(g.off), _p(g.col), _p(new_id), _p(off), _p(col))
    return Graph(off, col[:nnz].copy(), g.name)


def rmat_edges(scale: int, m: int, seed: int, abc=RMAT_ABC, n_limit: int = 0):
    lib = _load()
    src = np.empty(max(m, 1), dtype=np.int32)
    dst = np.empty(max(m, 1), dtype=np.int32)
    rc = lib.gen_rmat_edges(scale, m, abc[0], abc[1], abc[2], seed, n_limit, _p(src), _p(dst))
    if rc != 0:
        raise RuntimeError("R-MAT rejection sampling did not converge")
    return src[:m], dst[:m]


def rmat_graph(scale: int, edge_factor: int, seed: int, abc=RMAT_ABC, n: int | None = None,
               lcc: bool = True) -> Graph:
    """R-MAT over ids [0, 2^scale) (or [0, n) with ids >= n redrawn),
    m = edge_factor * (number of ids) edges, cleaned, LCC kept and renumbered."""
    nv = (1 << scale) if n is None else int(n)
    m = edge_factor * nv
    src, dst = rmat_edges(scale, m, seed, abc, 0 if n is None else nv)
    g = clean_csr(nv, src, dst)
    if lcc:
        g = largest_component(g)
    g.name = f"rmat-s{scale}-ef{edge_factor}-seed{seed}" + ("" if n is None else f"-n{nv}")
    return g


def chung_lu_graph(n: int, mean_degree: float, gamma: float, seed: int, lcc: bool = False) -> Graph:
    """Chung-Lu with m = mean_degree*n/2 edges drawn i.i.d. proportional to
    (i+1)^(-1/(gamma-1)); all vertices kept unless lcc."""
    lib = _load()
    m = int(round(mean_degree * n / 2))
    src = np.empty(max(m, 1), dtype=np.int32)
    dst = np.empty(max(m, 1), dtype=np.int32)
    if lib.gen_chung_lu_edges(n, m, gamma, seed, _p(src), _p(dst)) != 0:
        raise RuntimeError("Chung-Lu generation failed")
    g = clean_csr(n, src[:m], dst[:m])
    if lcc:
        g = largest_component(g)
    g.name = f"chunglu-n{n}-deg{mean_degree:g}-g{gamma:g}-seed{seed}"
    return g


def degree_order(g: Graph) -> np.ndarray:
    """order[r] = vertex id of rank r: degree descending, ties by smaller id."""
    lib = _load()
    order = np.empty(max(g.n, 1), dtype=np.int32)
    lib.gen_degree_order(g.n, _p(g.off), _p(order))
    return order[: g.n]


@dataclass
class DiGraph:
    """Directed graph: out-arcs (off, col) and their transpose (off_in, col_in);
    rows sorted, no self-loops, no duplicate arcs."""
    off: np.ndarray
    col: np.ndarray
    off_in: np.ndarray
    col_in: np.ndarray
    name: str = ""

    @property
    def n(self) -> int:
        return int(self.off.shape[0] - 1)

    @property
    def arcs(self) -> int:
        return int(self.col.shape[0])


def _rows(n: int, src: np.ndarray, dst: np.ndarray):
    key = np.unique(src.astype(np.int64) * n + dst.astype(np.int64))   # sorted by (src, dst), no duplicates
    s, d = (key // n).astype(np.int64), (key % n).astype(np.int32)
    off = np.zeros(n + 1, dtype=np.int64)
    np.add.at(off, s + 1, 1)
    return np.cumsum(off), d


def directed_csr(n: int, src, dst, name: str = "") -> DiGraph:
    """Arcs src[i] -> dst[i]: self-loops and duplicate arcs dropped; the
    transpose is built too."""
    src = np.asarray(src, dtype=np.int64)
    dst = np.asarray(dst, dtype=np.int64)
    keep = src != dst
    src, dst = src[keep], dst[keep]
    off, col = _rows(n, src, dst)
    off_in, col_in = _rows(n, dst, src)
    return DiGraph(off, col, off_in, col_in, name)


def rmat_digraph(scale: int, edge_factor: int, seed: int) -> DiGraph:
    """R-MAT arcs (the same draws as ``rmat_graph``) kept directed: 2^scale
    vertices, edge_factor * 2^scale arcs before dropping self-loops and
    duplicates; all vertices kept."""
    n = 1 << scale
    src, dst = rmat_edges(scale, edge_factor * n, seed)
    return directed_csr(n, src, dst, f"rmat-directed{scale}-{edge_factor}-{seed}")


def directed_degree_order(g: DiGraph) -> np.ndarray:
    """order[r] = vertex of rank r: in-degree + out-degree descending, ties by
    smaller id (the directed reading of Sec. 6.1's degree order)."""
    deg = np.diff(g.off) + np.diff(g.off_in)
    return np.lexsort((np.arange(g.n), -deg)).astype(np.int32)


def uniform_pairs(n: int, q: int, seed: int) -> np.ndarray:
    """int32[q, 2], s and t i.i.d. uniform on [0, n) (s == t allowed)."""
    lib = _load()
    pairs = np.empty(max(2 * q, 2), dtype=np.int32)
    if q > 0:
        lib.gen_uniform_pairs(n, q, seed, _p(pairs))
    return pairs[: 2 * q].reshape(q, 2)


def _splitmix64(z: np.ndarray) -> np.ndarray:
    """SplitMix64 output function (Steele, Lea, Flood 2014) on uint64 arrays."""
    with np.errstate(over="ignore"):
        z = z + np.uint64(0x9E3779B97F4A7C15)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        return z ^ (z >> np.uint64(31))


def edge_weights(g: Graph, lo: int, hi: int, seed: int) -> np.ndarray:
    """uint8 weight per arc of g, uniform on [lo, hi] per undirected edge:
    the arcs u -> v and v -> u hash the same key (min, max, seed), so both
    directions carry one weight (the paper's weighted inputs draw 1..7
    uniformly per edge, Sec. 6.1)."""
    if not 1 <= lo <= hi <= 255:
        raise ValueError("weights must lie in [1, 255]")
    src = np.repeat(np.arange(g.n, dtype=np.uint64), np.diff(g.off).astype(np.int64))
    dst = g.col.astype(np.uint64)
    a, b = np.minimum(src, dst), np.maximum(src, dst)
    with np.errstate(over="ignore"):
        key = (a << np.uint64(32)) ^ b ^ (np.uint64(seed) * np.uint64(0xD1B54A32D192ED03))
    h = _splitmix64(key)
    return (np.uint64(lo) + h % np.uint64(hi - lo + 1)).astype(np.uint8)


def uniform_int(seed: int, stream: int, i: int, lo: int, hi: int) -> int:
    return int(_load().gen_uniform_int(seed, stream, i, lo, hi))


def uniform01(seed: int, stream: int, i: int) -> float:
    return float(_load().gen_uniform01(seed, stream, i))


# ------------------------------------------------------------------ workloads
def small_graph_size(i: int) -> int:
    """Vertex count of small graph i of the batched workload: round(2^U(10,16))."""
    return int(_load().gen_log_uniform_size(100 + i, 10.0, 16.0))


def small_graph(i: int) -> Graph:
    """Graph i (seed 100+i) of the 2,000-graph batch: even i R-MAT edge factor 8
    over n_i ids (ids >= n_i redrawn) then LCC; odd i Chung-Lu gamma 2.3, mean
    degree 10, all vertices kept."""
    n_i = small_graph_size(i)
    seed = 100 + i
    if i % 2 == 0:
        scale = max(1, math.ceil(math.log2(n_i)))
        g = rmat_graph(scale, 8, seed, n=n_i, lcc=True)
    else:
        g = chung_lu_graph(n_i, 10.0, 2.3, seed)
    g.name = f"small{i}-" + g.name
    return g


def workload(name: str) -> Graph:
    """Named workloads:

    * ``rmat12``     R-MAT scale 12, edge factor 8, seed 1, LCC
    * ``chunglu20``  Chung-Lu 2^20 vertices, mean degree 16, gamma 2.1, seed 2
    * ``rmat22``     R-MAT scale 22, edge factor 16, seed 3, LCC
    """
    if name == "rmat12":
        return rmat_graph(12, 8, 1)
    if name == "chunglu20":
        return chung_lu_graph(1 << 20, 16.0, 2.1, 2)
    if name == "rmat22":
        return rmat_graph(22, 16, 3)
    if name.startswith("rmat") and "-" in name:  # rmatS-EF-SEED
        s, ef, seed = name[4:].split("-")
        return rmat_graph(int(s), int(ef), int(seed))
    if name.startswith("chunglu") and "-" in name:  # chungluN-DEG-GAMMA-SEED
        n, deg, gam, seed = name[7:].split("-")
        return chung_lu_graph(int(n), float(deg), float(gam), int(seed))
    raise KeyError(name)
