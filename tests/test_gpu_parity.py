"""GPU path vs the CPU oracle, element by element, through the C ABI.

Labels must be bit-exact as hub-sorted rows (hub rank, distance); query
answers must be bit-exact (integers, no tolerance).
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1906_12018_gb300 import graphs as G
from paper_1906_12018_gb300 import plb

from gpu_util import assert_labels_equal, gpu_build, gpu_query, host_labels, to_device
from test_oracle import apsp, tiny_graphs

pytestmark = pytest.mark.gpu


def orders_for(g, seed=3):
    rng = np.random.default_rng(seed)
    return [G.degree_order(g), np.arange(g.n, dtype=np.int32), rng.permutation(g.n).astype(np.int32)]


@pytest.mark.parametrize("name,g", tiny_graphs(), ids=lambda x: x if isinstance(x, str) else "")
def test_tiny_graphs_match_definition(name, g):
    for order in orders_for(g):
        ref = O.chhl(g.off, g.col, order)
        lab = gpu_build(g, order)
        assert_labels_equal(lab, ref, name)


@pytest.fixture(scope="module")
def rmat12():
    g = G.workload("rmat12")
    order = G.degree_order(g)
    return g, order, O.pll(g.off, g.col, order)


def test_rmat12_labels_bit_exact(rmat12):
    g, order, ref = rmat12
    lab = gpu_build(g, order)
    assert_labels_equal(lab, ref, "rmat12")
    assert lab.max_dist == ref.max_dist


def test_rmat12_queries_bit_exact(rmat12):
    g, order, ref = rmat12
    lab = gpu_build(g, order)
    pairs = G.uniform_pairs(g.n, 10_000, 1)
    got = gpu_query(lab, pairs)
    assert np.array_equal(got, O.query(ref, pairs))
    D = apsp(g)
    want = D[pairs[:, 0], pairs[:, 1]]
    assert np.array_equal(got, np.where(np.isfinite(want), want, -1).astype(np.int64))


def test_rmat12_rounds_match_vcpll(rmat12):
    """Per round: the same number of new labels as Alg. 3 restated on the CPU,
    and the same number of distinct checked candidates."""
    g, order, _ = rmat12
    vc = O.vcpll(g.off, g.col, order)
    lab = gpu_build(g, order)
    st = lab.stats()
    assert st["rounds"] == vc.rounds
    assert st["accepted"] == [int(x) for x in vc.round_stats[1:vc.rounds + 1, 2]]
    assert st["unique_candidates"] == int(vc.round_stats[:, 1].sum())


def test_all_tiers_bit_exact(rmat12):
    """Tiny table capacities push vertices through the block tier, split their
    candidates into many hub-range passes, and leave rows too long for the
    shared-memory map to the global probe table; the labels must not change."""
    g, order, ref = rmat12
    lab = gpu_build(g, order, warp_cand_cap=32, warp_label_cap=16, block_cand_cap=64, block_label_cap=24,
                    block_threads=64)
    assert_labels_equal(lab, ref, "forced tiers")
    st = lab.stats()
    assert st["tier_vertices"][0] > 0 and st["tier_vertices"][1] > 0, st["tier_vertices"]
    assert max(np.diff(host_labels(lab)[0])) > 64          # some rows skip the map


def test_edge_cases():
    # no vertices
    g0 = G.from_edges(0, [])
    lab = gpu_build(g0, np.zeros(0, np.int32))
    assert lab.total == 0 and lab.n == 0
    # single vertex, isolated vertices
    for n in (1, 7):
        g = G.from_edges(n, [])
        order = G.degree_order(g)
        lab = gpu_build(g, order)
        assert_labels_equal(lab, O.pll(g.off, g.col, order), f"isolated{n}")
        assert np.array_equal(gpu_query(lab, [[0, n - 1], [0, 0]]), [0 if n == 1 else -1, 0])
    # star, complete graph, path reaching the largest distance 254
    cases = [G.from_edges(40, [(0, i) for i in range(1, 40)]),
             G.from_edges(25, [(i, j) for i in range(25) for j in range(i + 1, 25)]),
             G.from_edges(255, [(i, i + 1) for i in range(254)])]
    for g in cases:
        order = G.degree_order(g)
        lab = gpu_build(g, order)
        assert_labels_equal(lab, O.pll(g.off, g.col, order))
    # path in position order: vertex i has every j <= i as a hub, up to d = 254
    order = np.arange(255, dtype=np.int32)
    lab = gpu_build(cases[-1], order)
    assert_labels_equal(lab, O.pll(cases[-1].off, cases[-1].col, order))
    assert lab.max_dist == 254 and lab.rounds == 255


def test_distance_overflow_is_an_error():
    g = G.from_edges(300, [(i, i + 1) for i in range(299)])
    with pytest.raises(plb.PLBError) as e:
        gpu_build(g, np.arange(300, dtype=np.int32))
    assert e.value.code == plb.PLB_ERR_DIST_OVERFLOW


def _bad_build(off, col, order):
    dev = torch.device("cuda:0")
    rp = torch.tensor(off, dtype=torch.int64, device=dev)
    c = torch.tensor(col, dtype=torch.int32, device=dev)
    o = torch.tensor(order, dtype=torch.int32, device=dev)
    with pytest.raises(plb.PLBError) as e:
        plb.build(rp, c, o)
    return e.value.code


def test_invalid_inputs_rejected():
    ok_off, ok_col = [0, 1, 3, 4], [1, 0, 2, 1]           # path 0-1-2
    assert _bad_build([0, 1, 3, 4], [1, 0, 2, 0], [0, 1, 2]) == plb.PLB_ERR_INVALID   # asymmetric
    assert _bad_build([0, 1, 2, 3], [1, 0, 0], [0, 1, 2]) == plb.PLB_ERR_INVALID      # asymmetric: arc 2->0 alone
    assert _bad_build([0, 1, 3, 4], [1, 2, 0, 1], [0, 1, 2]) == plb.PLB_ERR_INVALID   # unsorted row
    assert _bad_build([0, 2, 4, 5], [0, 1, 0, 2, 1], [0, 1, 2]) == plb.PLB_ERR_INVALID  # self-loop
    assert _bad_build([0, 1, 3, 4], [1, 0, 7, 1], [0, 1, 2]) == plb.PLB_ERR_INVALID   # out of range
    assert _bad_build([0, 1, 4, 5], [1, 0, 2, 2, 1], [0, 1, 2]) == plb.PLB_ERR_INVALID  # duplicate
    assert _bad_build([0, 3, 3, 4], ok_col, [0, 1, 2]) == plb.PLB_ERR_INVALID        # bad row_ptr
    assert _bad_build(ok_off, ok_col, [0, 1, 1]) == plb.PLB_ERR_INVALID               # order not a permutation
    assert _bad_build(ok_off, ok_col, [0, 1, 5]) == plb.PLB_ERR_INVALID               # order out of range


def test_degree_order_matches_generator(rmat12):
    for g in (rmat12[0], G.small_graph(1), G.from_edges(5, [(0, 1)])):
        rp, _, _ = to_device(g, np.zeros(g.n, np.int32))
        got = plb.degree_order(rp)
        torch.cuda.synchronize()
        assert np.array_equal(got.cpu().numpy(), G.degree_order(g))


def test_batch_equals_single_and_oracle():
    gs = [G.small_graph(i) for i in range(10)] + [G.from_edges(3, [(0, 1)]), G.workload("rmat12")]
    orders = [G.degree_order(g) for g in gs]
    dev = [to_device(g, o) for g, o in zip(gs, orders)]
    batch = plb.build_batch(dev)
    for i, (g, o) in enumerate(zip(gs, orders)):
        single = plb.build(*dev[i])
        a = host_labels(batch[i])
        b = host_labels(single)
        for x, y in zip(a, b):
            assert np.array_equal(x, y), i
        if g.n <= 40_000:
            ref = O.pll(g.off, g.col, o)
            assert_labels_equal(batch[i], ref, f"batch part {i}")
        pairs = G.uniform_pairs(g.n, 500, 7 + i)
        assert np.array_equal(gpu_query(batch[i], pairs), gpu_query(single, pairs))


def test_query_multi_matches_single(rmat12):
    g1, o1, _ = rmat12
    g2 = G.small_graph(3)
    o2 = G.degree_order(g2)
    l1 = gpu_build(g1, o1)
    l2 = gpu_build(g2, o2)
    rng = np.random.default_rng(5)
    q = 4000
    sidx = rng.integers(0, 2, q).astype(np.int32)
    sidx[:3] = [5, -1, 2]  # bad set indices
    n = np.where(sidx == 1, g2.n, g1.n)
    pairs = (rng.random((q, 2)) * n[:, None]).astype(np.int32)
    got = plb.query_multi([l1, l2], torch.from_numpy(sidx).cuda(), torch.from_numpy(pairs).cuda())
    torch.cuda.synchronize()
    got = got.cpu().numpy()
    assert np.all(got[:3] == plb.PLB_BAD_PAIR)
    for k, lab in ((0, l1), (1, l2)):
        m = sidx == k
        assert np.array_equal(got[m], gpu_query(lab, pairs[m]))
    bad = gpu_query(l1, [[0, g1.n], [-1, 0]])
    assert np.all(bad == plb.PLB_BAD_PAIR)


@pytest.fixture(scope="module")
def chunglu20():
    g = G.workload("chunglu20")
    order = G.degree_order(g)
    lab = gpu_build(g, order)
    return g, order, lab


def test_chunglu20_sampled_rows_match_definition(chunglu20):
    """Full-size bench graph, default launch configuration: 64 sampled rows
    equal Def. 2 computed one vertex at a time."""
    g, order, lab = chunglu20
    off, hub, dist = host_labels(lab)
    rng = np.random.default_rng(20)
    deg = g.degrees()
    picks = list(rng.choice(g.n, 48, replace=False)) + list(order[:8]) + list(np.argsort(-deg)[100:108])
    for v in picks:
        h, d = O.chhl_row(g.off, g.col, order, int(v))
        a, b = int(off[v]), int(off[v + 1])
        assert np.array_equal(hub[a:b], h), v
        assert np.array_equal(dist[a:b], d), v


def test_chunglu20_sampled_queries_match_bfs(chunglu20):
    g, order, lab = chunglu20
    rng = np.random.default_rng(21)
    srcs = rng.choice(g.n, 12, replace=False)
    pairs = []
    for s in srcs:
        t = rng.choice(g.n, 500, replace=False)
        pairs.append(np.stack([np.full(500, s), t], 1))
    pairs = np.concatenate(pairs).astype(np.int32)
    got = gpu_query(lab, pairs)
    for i, s in enumerate(srcs):
        D = O.bfs(g.off, g.col, int(s))
        assert np.array_equal(got[i * 500:(i + 1) * 500], D[pairs[i * 500:(i + 1) * 500, 1]])


def test_chunglu20_batched_equals_unbatched(chunglu20):
    """Alg. 4 with four batches of 2^18 hubs gives the same labels (compared
    on the device, every entry)."""
    g, order, lab = chunglu20
    lab_b = gpu_build(g, order, batch_hubs=1 << 18)
    assert lab_b.total == lab.total
    for x, y in zip(lab.device_arrays(), lab_b.device_arrays()):
        assert torch.equal(x, y)
    lab_b.free()


def test_chunglu20_invariants(chunglu20):
    g, order, lab = chunglu20
    off, hub, dist = host_labels(lab)
    rank = np.empty(g.n, dtype=np.int64)
    rank[order] = np.arange(g.n)
    lens = np.diff(off)
    last = off[1:] - 1
    assert np.all(lens >= 1)
    assert np.array_equal(hub[last].astype(np.int64), rank)           # (v, 0) closes every row
    assert np.all(dist[last] == 0)
    row = np.repeat(np.arange(g.n), lens)
    assert np.all(hub.astype(np.int64) <= rank[row])                  # hierarchy
    inner = np.ones(hub.shape[0], bool)
    inner[off[:-1]] = False
    assert np.all(np.diff(hub.astype(np.int64))[inner[1:]] > 0)       # strictly increasing rows


@pytest.mark.slow
def test_chunglu20_full_oracle(chunglu20):
    """Every label of the 2^20-vertex graph against the sequential PLL oracle."""
    g, order, lab = chunglu20
    ref = O.pll(g.off, g.col, order)
    assert_labels_equal(lab, ref, "chunglu20")


def test_graph_mode_bit_exact(rmat12):
    """The round loop as one captured CUDA graph gives the same labels, the
    same per-round counts, and handles the terminating round on the device."""
    g, order, ref = rmat12
    lab = gpu_build(g, order, use_graph=1)
    assert_labels_equal(lab, ref, "graph mode")
    host = gpu_build(g, order).stats()
    st = lab.stats()
    assert st["rounds"] == host["rounds"] and st["accepted"] == host["accepted"]
    assert st["unique_round"] == host["unique_round"]
    for gi in (G.small_graph(2), G.from_edges(40, [(0, i) for i in range(1, 40)])):
        o = G.degree_order(gi)
        assert_labels_equal(gpu_build(gi, o, use_graph=1), O.pll(gi.off, gi.col, o), "graph mode small")


def test_graph_mode_after_a_large_first_round():
    """K_1500 accepts 1.1M labels in round 1 (host-driven), more than the
    graph's minimum label capacity (2^20): the graph is sized from them and
    finishes the build; labels unchanged."""
    n = 1500
    g = G.from_edges(n, [(i, j) for i in range(n) for j in range(i + 1, n)])
    order = np.arange(n, dtype=np.int32)
    lab = gpu_build(g, order, use_graph=1)
    assert lab.total == n * (n + 1) // 2
    assert lab.rounds == gpu_build(g, order).rounds
    assert_labels_equal(lab, O.pll(g.off, g.col, order), "K1500")


def test_graph_mode_capacity_mid_build():
    """A star of 1536 leaves whose centre is ranked last: round 1 gives the
    centre every leaf (1536 labels), round 2 gives every leaf each higher
    ranked leaf at distance 2 (any witness path is 4 long), 1.18M labels,
    which stops the graph in round 2; it resumes with round 3."""
    leaves = 1536
    n = leaves + 1
    g = G.from_edges(n, [(i, leaves) for i in range(leaves)])
    order = np.arange(n, dtype=np.int32)
    lab = gpu_build(g, order, use_graph=1)
    pairs = leaves * (leaves - 1) // 2
    assert lab.total == n + leaves + pairs
    st = lab.stats()
    assert st["reruns"] >= 1 and lab.rounds == gpu_build(g, order).rounds
    assert st["accepted"][:2] == [leaves, pairs]
    assert_labels_equal(lab, O.pll(g.off, g.col, order), "star, centre last")


def test_graph_mode_distance_overflow():
    g = G.from_edges(300, [(i, i + 1) for i in range(299)])
    with pytest.raises(plb.PLBError) as e:
        gpu_build(g, np.arange(300, dtype=np.int32), use_graph=1)
    assert e.value.code == plb.PLB_ERR_DIST_OVERFLOW


def test_largest_vertex_count():
    """n = 2^24 - 1, the most vertices the 24-bit hub field admits: a double
    star (centres 0 and 1 joined, leaf i on centre i mod 2).  Even leaves get
    (0,1); odd leaves (1,1) in round 1 and (0,2) in round 2 (no hub common to
    the leaf and 0 yet); every vertex its (v,0)."""
    n = (1 << 24) - 1
    leaves = np.arange(2, n, dtype=np.int32)
    src = np.concatenate([np.array([0], np.int32), leaves])
    dst = np.concatenate([np.array([1], np.int32), (leaves % 2).astype(np.int32)])
    g = G.clean_csr(n, src, dst)
    order = G.degree_order(g)
    assert np.array_equal(order[:3], [0, 1, 2]) and order[-1] == n - 1
    lab = gpu_build(g, order)
    n_even, n_odd = (n - 1) // 2, (n - 2) // 2
    assert lab.total == 1 + 2 + 2 * n_even + 3 * n_odd
    assert lab.max_dist == 2 and lab.rounds == 3
    off_d, hub_d, dist_d = lab.device_arrays()
    for v, want in ((0, [(0, 0)]), (1, [(0, 1), (1, 0)]), (n - 1, [(0, 1), (n - 1, 0)]),
                    (n - 2, [(0, 2), (1, 1), (n - 2, 0)])):
        a, b = int(off_d[v]), int(off_d[v + 1])
        got = list(zip(hub_d[a:b].cpu().numpy().astype(np.int64).tolist(), dist_d[a:b].cpu().numpy().tolist()))
        assert got == want, (v, got)
    pairs = np.array([[n - 1, n - 2], [n - 2, 3], [n - 1, 2], [n - 1, n - 1], [0, n - 2], [1, n - 1]], np.int32)
    assert gpu_query(lab, pairs).tolist() == [3, 2, 2, 0, 2, 2]
    lab.free()


def test_batched_labels_equal_unbatched(rmat12):
    """Alg. 4: hubs propagated in rank batches give the canonical labels of
    Alg. 3 for any batch size, with the same number of labels per distance."""
    g, order, ref = rmat12
    base = gpu_build(g, order).stats()
    r = base["rounds"]
    for b in (7, 64, 1000):
        lab = gpu_build(g, order, batch_hubs=b)
        assert_labels_equal(lab, ref, f"batch {b}")
        acc = lab.stats()["accepted"]
        assert acc[:r] == base["accepted"] and not any(acc[r:]), b
    lab = gpu_build(g, order, batch_hubs=64, use_graph=1)  # graph mode is off in batches
    assert_labels_equal(lab, ref, "batch 64 graph")


@pytest.mark.parametrize("name,g", tiny_graphs(), ids=lambda x: x if isinstance(x, str) else "")
def test_tiny_graphs_batch_of_one_hub(name, g):
    """A batch of one hub is PLL's one root at a time (Sec. 4.2)."""
    for order in orders_for(g):
        ref = O.chhl(g.off, g.col, order)
        assert_labels_equal(gpu_build(g, order, batch_hubs=1), ref, name)
