"""Weighted labeling (Sec. 5.1) on the GPU against the weighted oracle,
element by element, through the C ABI (plb_build_weighted, then
plb_query_batch on the weighted labels)."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1906_12018_gb300 import graphs as G
from paper_1906_12018_gb300 import plb

from gpu_util import assert_labels_equal, gpu_build, gpu_query, host_labels
from test_oracle_weighted import tiny_wgraphs, wgraph

pytestmark = pytest.mark.gpu


def dev(a, dtype):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=dtype)).cuda()


def gpu_build_weighted(g, wt, order, **opts):
    return plb.build_weighted(dev(g.off, np.int64), dev(g.col, np.int32), dev(wt, np.uint8), dev(order, np.int32),
                              **opts)


FORCED = dict(warp_cand_cap=32, warp_label_cap=16, block_cand_cap=64, block_label_cap=24, block_threads=64)


@pytest.mark.parametrize("name,g,wt", tiny_wgraphs(), ids=lambda x: x if isinstance(x, str) else "")
def test_tiny_weighted_match_definition(name, g, wt):
    rng = np.random.default_rng(3)
    for order in (G.degree_order(g), np.arange(g.n, dtype=np.int32), rng.permutation(g.n).astype(np.int32)):
        ref = O.chhl_weighted(g.off, g.col, wt, order)
        assert_labels_equal(gpu_build_weighted(g, wt, order), ref, name)


@pytest.fixture(scope="module")
def rmat12w():
    g = G.workload("rmat12")
    wt = G.edge_weights(g, 1, 7, 1)
    order = G.degree_order(g)
    return g, wt, order, O.pll_weighted(g.off, g.col, wt, order)


def test_weighted_rmat12_labels_and_queries(rmat12w):
    g, wt, order, ref = rmat12w
    L = gpu_build_weighted(g, wt, order)
    assert_labels_equal(L, ref, "rmat12 weighted")
    assert L.stats()["rounds"] >= int(ref.max_dist)  # one round per distance
    pairs = G.uniform_pairs(g.n, 10000, 1)
    assert np.array_equal(gpu_query(L, pairs), O.query(ref, pairs))
    for s in (0, 5, 777):
        p = np.stack([np.full(g.n, s), np.arange(g.n)], 1).astype(np.int32)
        assert np.array_equal(gpu_query(L, p), O.dijkstra(g.off, g.col, wt, s))


def test_weighted_all_tiers(rmat12w):
    g, wt, order, ref = rmat12w
    L = gpu_build_weighted(g, wt, order, **FORCED)
    assert_labels_equal(L, ref, "forced tiers")
    assert L.stats()["tier_vertices"][1] > 0


def test_unit_weights_equal_the_unweighted_build():
    g = G.rmat_graph(13, 8, 6)
    order = G.degree_order(g)
    W = host_labels(gpu_build_weighted(g, np.ones(g.col.shape[0], np.uint8), order))
    U = host_labels(gpu_build(g, order))
    for x, y in zip(W, U):
        assert np.array_equal(x, y)


def test_constant_weight_scales_the_unweighted_build():
    """Every weight 7: rounds 7, 14, ... carry the labels, the six rounds in
    between have no receivers; hubs as unweighted, distances times 7."""
    g = G.rmat_graph(12, 8, 2)
    order = G.degree_order(g)
    off, hub, dist = host_labels(gpu_build_weighted(g, np.full(g.col.shape[0], 7, np.uint8), order))
    uo, uh, ud = host_labels(gpu_build(g, order))
    assert np.array_equal(off, uo) and np.array_equal(hub, uh)
    assert np.array_equal(dist.astype(np.int32), 7 * ud.astype(np.int32))


def test_wide_weights_and_distance_overflow():
    """Weights up to 60 (a 61-slot frontier ring); where a distance passes 254
    both sides refuse."""
    g = G.rmat_graph(9, 4, 3)
    order = G.degree_order(g)
    for lo, hi, seed in ((1, 60, 4), (30, 60, 5)):
        wt = G.edge_weights(g, lo, hi, seed)
        try:
            ref = O.pll_weighted(g.off, g.col, wt, order)
        except OverflowError:
            with pytest.raises(plb.PLBError) as e:
                gpu_build_weighted(g, wt, order)
            assert e.value.code == plb.PLB_ERR_DIST_OVERFLOW
            continue
        assert_labels_equal(gpu_build_weighted(g, wt, order), ref, f"weights {lo}..{hi}")


def test_weighted_chunglu16_with_isolated_vertices():
    g = G.chung_lu_graph(1 << 16, 16.0, 2.1, 2)
    wt = G.edge_weights(g, 1, 7, 2)
    order = G.degree_order(g)
    assert np.any(np.diff(g.off) == 0)
    assert_labels_equal(gpu_build_weighted(g, wt, order), O.pll_weighted(g.off, g.col, wt, order), "chunglu16 w")


def test_weighted_chunglu20_sampled_rows():
    """The benchmark's weighted workload (Chung-Lu 2^20, mean degree 16,
    gamma 2.1, seed 2, weights 1..7 seed 2) with the default options: rows
    of sampled and of the highest-degree vertices against Def. 2, queries
    against Dijkstra from a few sources."""
    g = G.workload("chunglu20")
    wt = G.edge_weights(g, 1, 7, 2)
    order = G.degree_order(g)
    L = gpu_build_weighted(g, wt, order)
    off, hub, dist = host_labels(L)
    rng = np.random.default_rng(20)
    deg = np.diff(g.off)
    for v in list(rng.choice(g.n, 16, replace=False)) + list(np.argsort(-deg)[:4]):
        h, d = O.chhl_row_weighted(g.off, g.col, wt, order, int(v))
        assert np.array_equal(hub[off[v]:off[v + 1]], h) and np.array_equal(dist[off[v]:off[v + 1]], d), v
    for s in rng.choice(g.n, 2, replace=False):
        p = np.stack([np.full(g.n, s), np.arange(g.n)], 1).astype(np.int32)
        assert np.array_equal(gpu_query(L, p), O.dijkstra(g.off, g.col, wt, int(s)))


def test_weighted_invalid_inputs():
    g, wt = wgraph(3, [(0, 1, 2), (1, 2, 3)])
    order = np.arange(3, dtype=np.int32)
    L = gpu_build_weighted(g, wt, order)
    assert L.total == 3 + 2 + 1
    bad0 = wt.copy()
    bad0[0] = 0
    asym = wt.copy()
    asym[0] = 5          # arc 0 -> 1 differs from 1 -> 0
    for w in (bad0, asym):
        with pytest.raises(plb.PLBError) as e:
            gpu_build_weighted(g, w, order)
        assert e.value.code == plb.PLB_ERR_INVALID
    with pytest.raises(plb.PLBError) as e:   # a zero weight is refused even without validation
        gpu_build_weighted(g, bad0, order, validate=0)
    assert e.value.code == plb.PLB_ERR_INVALID
    with pytest.raises(ValueError):
        gpu_build_weighted(g, wt[:-1], order)
