"""Directed labeling (Sec. 5.1) on the GPU against the directed oracle,
element by element, through the C ABI (plb_build_directed,
plb_query_directed)."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1906_12018_gb300 import graphs as G
from paper_1906_12018_gb300 import plb

from gpu_util import assert_labels_equal, host_labels
from test_oracle_directed import tiny_digraphs

pytestmark = pytest.mark.gpu


def dev(a, dtype):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=dtype)).cuda()


def gpu_build_directed(g, order, **opts):
    return plb.build_directed(dev(g.off, np.int64), dev(g.col, np.int32), dev(order, np.int32), **opts)


def orders_for(g, seed=3):
    rng = np.random.default_rng(seed)
    return [G.directed_degree_order(g), np.arange(g.n, dtype=np.int32), rng.permutation(g.n).astype(np.int32)]


@pytest.mark.parametrize("name,g", tiny_digraphs(), ids=lambda x: x if isinstance(x, str) else "")
def test_tiny_digraphs_match_definition(name, g):
    for order in orders_for(g):
        ref_in, ref_out = O.chhl_directed(g.off, g.col, g.off_in, g.col_in, order)
        lin, lout = gpu_build_directed(g, order)
        assert_labels_equal(lin, ref_in, name + " in")
        assert_labels_equal(lout, ref_out, name + " out")


@pytest.fixture(scope="module")
def rmat12d():
    g = G.rmat_digraph(12, 8, 1)
    order = G.directed_degree_order(g)
    ref_in, ref_out = O.pll_directed(g.off, g.col, g.off_in, g.col_in, order)
    return g, order, ref_in, ref_out


def test_directed_rmat12_labels_and_queries(rmat12d):
    g, order, ref_in, ref_out = rmat12d
    lin, lout = gpu_build_directed(g, order)
    assert_labels_equal(lin, ref_in, "rmat12 directed in")
    assert_labels_equal(lout, ref_out, "rmat12 directed out")
    pairs = G.uniform_pairs(g.n, 20000, 5)
    got = plb.query_directed(lout, lin, dev(pairs, np.int32))
    torch.cuda.synchronize()
    assert np.array_equal(got.cpu().numpy(), O.query_directed(ref_out, ref_in, pairs))
    # d(s -> t) against BFS from a few sources
    for s in (0, 17, 1000):
        D = O.bfs(g.off, g.col, s)
        p = np.stack([np.full(g.n, s), np.arange(g.n)], 1).astype(np.int32)
        assert np.array_equal(plb.query_directed(lout, lin, dev(p, np.int32)).cpu().numpy(), D)


def test_directed_all_tiers(rmat12d):
    """Tiny tables push vertices through the block tier and its hub-range
    passes in both directions."""
    g, order, ref_in, ref_out = rmat12d
    lin, lout = gpu_build_directed(g, order, warp_cand_cap=32, warp_label_cap=16, block_cand_cap=64,
                                   block_label_cap=24, block_threads=64)
    assert_labels_equal(lin, ref_in, "forced in")
    assert_labels_equal(lout, ref_out, "forced out")
    assert lin.stats()["tier_vertices"][1] > 0 and lout.stats()["tier_vertices"][1] > 0


def test_symmetric_digraph_equals_undirected():
    g = G.rmat_graph(11, 8, 4)
    order = G.degree_order(g)
    d = G.directed_csr(g.n, np.repeat(np.arange(g.n), np.diff(g.off)), g.col)
    lin, lout = gpu_build_directed(d, order)
    u = plb.build(dev(g.off, np.int64), dev(g.col, np.int32), dev(order, np.int32))
    ref = host_labels(u)
    for L in (lin, lout):
        for x, y in zip(host_labels(L), ref):
            assert np.array_equal(x, y)


def test_directed_sampled_rows_rmat16():
    g = G.rmat_digraph(16, 16, 2)
    order = G.directed_degree_order(g)
    lin, lout = gpu_build_directed(g, order)
    oi, hi, di = host_labels(lin)
    oo, ho, do = host_labels(lout)
    rng = np.random.default_rng(16)
    deg = np.diff(g.off) + np.diff(g.off_in)
    for v in list(rng.choice(g.n, 24, replace=False)) + list(np.argsort(-deg)[:4]):
        h, d = O.chhl_row(g.off_in, g.col_in, order, int(v))      # L_in(v): shortest x -> v paths
        assert np.array_equal(hi[oi[v]:oi[v + 1]], h) and np.array_equal(di[oi[v]:oi[v + 1]], d), v
        h, d = O.chhl_row(g.off, g.col, order, int(v))            # L_out(v)
        assert np.array_equal(ho[oo[v]:oo[v + 1]], h) and np.array_equal(do[oo[v]:oo[v + 1]], d), v


def test_directed_invalid_inputs():
    off, col = [0, 1, 2, 2], [1, 2]                               # 0 -> 1 -> 2 (no reverse arcs: fine)
    lin, lout = plb.build_directed(dev(off, np.int64), dev(col, np.int32), dev([0, 1, 2], np.int32))
    assert lin.total == 3 + 2 + 1 and lout.total == 3
    for o_, c_ in (([0, 1, 2, 2], [0, 2]), ([0, 2, 2, 2], [2, 1]), ([0, 1, 2, 2], [1, 5])):
        with pytest.raises(plb.PLBError) as e:                    # self-loop, unsorted row, out of range
            plb.build_directed(dev(o_, np.int64), dev(c_, np.int32), dev([0, 1, 2], np.int32))
        assert e.value.code == plb.PLB_ERR_INVALID


def test_directed_bench_workload_sampled_rows():
    """The directed bench workload (R-MAT arcs kept directed, 2^20 vertices,
    edge factor 16, seed 3) with the default options: rows of sampled and of
    the highest-degree vertices against Def. 2 in both directions, and
    d(s -> t) against BFS from two sources."""
    g = G.rmat_digraph(20, 16, 3)
    order = G.directed_degree_order(g)
    lin, lout = gpu_build_directed(g, order)
    oi, hi, di = host_labels(lin)
    oo, ho, do = host_labels(lout)
    rng = np.random.default_rng(20)
    deg = np.diff(g.off) + np.diff(g.off_in)
    for v in list(rng.choice(g.n, 12, replace=False)) + list(np.argsort(-deg)[:3]):
        h, d = O.chhl_row(g.off_in, g.col_in, order, int(v))
        assert np.array_equal(hi[oi[v]:oi[v + 1]], h) and np.array_equal(di[oi[v]:oi[v + 1]], d), v
        h, d = O.chhl_row(g.off, g.col, order, int(v))
        assert np.array_equal(ho[oo[v]:oo[v + 1]], h) and np.array_equal(do[oo[v]:oo[v + 1]], d), v
    for s in rng.choice(g.n, 2, replace=False):
        p = np.stack([np.full(g.n, s), np.arange(g.n)], 1).astype(np.int32)
        got = plb.query_directed(lout, lin, dev(p, np.int32)).cpu().numpy()
        assert np.array_equal(got, O.bfs(g.off, g.col, int(s)))
