"""R-MAT scale 22 (edge factor 16, seed 3, LCC: 2.39M vertices, 64.2M edges,
1.8G labels), the largest workload and the serving one, at full size with
the default launch configuration: every row against the stored digests of
the oracle's full PLL run, about 2,000 rows stratified by rank and degree
against Def. 2, sampled queries against BFS, and the row invariants over
every label (checked on the device, in slices)."""
import json
import os
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O  # noqa: E402
from gpu_util import build_peak, gpu_build, gpu_query  # noqa: E402
from paper_1906_12018_gb300 import graphs as G  # noqa: E402

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
sys.path.insert(0, GOLDEN)
import label_digest as LD  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rmat22():
    g = G.workload("rmat22")
    order = G.degree_order(g)
    lab = gpu_build(g, order)
    yield g, order, lab
    lab.free()
    torch.cuda.empty_cache()


def test_rmat22_size(rmat22):
    g, order, lab = rmat22
    assert (g.n, g.m) == (2394833, 64152981)
    assert lab.total == 1799946086


def test_rmat22_build_peak_within_the_admission_footprint(rmat22):
    """The serving loop admits a build by its footprint model; on the
    largest graph the machine's measured peak stays inside it."""
    from paper_1906_12018_gb300.serve import build_footprint

    g, _, _ = rmat22
    m = build_peak(g)
    assert m["left"] == 0
    assert 0 < m["peak"] <= build_footprint(g.n, g.nnz) - m["inputs"], (m, build_footprint(g.n, g.nnz))


def stratified_rows(g, order, per=32, seed=22):
    """Rows to compare with Def. 2: the 512 highest-ranked vertices, `per`
    random vertices from each of 16 equal rank strata and from each of 16
    degree-quantile strata, and 512 uniform picks (2,048 distinct rows at
    most)."""
    rng = np.random.default_rng(seed)
    n = g.n
    picks = set(int(x) for x in order[:512])
    for s in range(16):
        lo, hi = s * n // 16, (s + 1) * n // 16
        picks.update(int(x) for x in order[rng.integers(lo, hi, per)])
    by_deg = np.argsort(g.degrees(), kind="stable")
    for s in range(16):
        lo, hi = s * n // 16, (s + 1) * n // 16
        picks.update(int(x) for x in by_deg[rng.integers(lo, hi, per)])
    picks.update(int(x) for x in rng.choice(n, 512, replace=False))
    return sorted(picks)


def test_rmat22_stratified_rows_match_definition(rmat22):
    """About 2,000 rows stratified by rank and degree equal Def. 2, each
    computed by its own BFS (the oracle's Def. 2 row function, run on host
    threads)."""
    from concurrent.futures import ThreadPoolExecutor

    g, order, lab = rmat22
    off_d, hub_d, dist_d = lab.device_arrays()
    off = off_d.cpu().numpy()
    rows = stratified_rows(g, order)
    assert len(rows) >= 1500
    with ThreadPoolExecutor(max_workers=os.cpu_count() or 4) as ex:
        want = list(ex.map(lambda v: O.chhl_row(g.off, g.col, order, v), rows))
    for v, (h, d) in zip(rows, want):
        a, b = int(off[v]), int(off[v + 1])
        assert np.array_equal(hub_d[a:b].cpu().numpy().astype(np.uint32), h), v
        assert np.array_equal(dist_d[a:b].cpu().numpy(), d), v


def test_rmat22_all_labels_equal_oracle_digests(rmat22):
    """Every row: the GPU labels digested per block of 2^16 rows equal the
    stored digests of the oracle's full PLL run on this graph
    (tests/golden/rmat22_labels.json, written by tests/golden/make_digests.py)."""
    path = os.path.join(GOLDEN, "rmat22_labels.json")
    if not os.path.exists(path):
        pytest.skip("oracle digests of rmat22 not recorded")
    with open(path) as f:
        want = json.load(f)
    g, order, lab = rmat22
    assert (g.n, g.m, lab.total) == (want["n"], want["m"], want["labels"])
    off, hub, dist = lab.to_host()
    got = LD.block_digests(off, hub, dist, want["block_rows"])
    bad = [i for i, (a, b) in enumerate(zip(got, want["blocks"])) if a != b]
    assert len(got) == len(want["blocks"]) and bad == []


def test_rmat22_sampled_queries_match_bfs(rmat22):
    g, order, lab = rmat22
    rng = np.random.default_rng(23)
    srcs = rng.choice(g.n, 3, replace=False)
    pairs = np.concatenate([np.stack([np.full(1000, s), rng.choice(g.n, 1000, replace=False)], 1)
                            for s in srcs]).astype(np.int32)
    got = gpu_query(lab, pairs)
    for i, s in enumerate(srcs):
        D = O.bfs(g.off, g.col, int(s))
        assert np.array_equal(got[i * 1000:(i + 1) * 1000], D[pairs[i * 1000:(i + 1) * 1000, 1]])


def test_rmat22_invariants_all_rows(rmat22):
    """(v, 0) closes every row, hubs outrank their row's vertex, rows strictly
    increase: over all 1.8G labels."""
    g, order, lab = rmat22
    off, hub, dist = lab.device_arrays()
    dev = off.device
    rank = torch.empty(g.n, dtype=torch.int64, device=dev)
    rank[torch.from_numpy(order.astype(np.int64)).to(dev)] = torch.arange(g.n, device=dev)
    last = off[1:] - 1
    assert bool(torch.all(off[1:] > off[:-1]))
    assert torch.equal(hub[last].long(), rank)
    assert bool(torch.all(dist[last] == 0))
    step = 1 << 27
    for a in range(0, lab.total, step):
        a = max(a - 1, 0)  # slices overlap by one entry: every adjacent pair is compared
        b = min(lab.total, a + 1 + step)
        q = torch.arange(a, b, device=dev)
        r = torch.searchsorted(off, q, right=True) - 1      # row of each entry
        assert bool(torch.all(hub[a:b].long() <= rank[r]))   # hierarchy
        if b - a > 1:
            same = r[1:] == r[:-1]
            inc = hub[a + 1:b].long() > hub[a:b - 1].long()
            assert bool(torch.all(inc | ~same))              # strictly increasing within rows
        del q, r


def test_rmat22_serving_results_identical_alone_and_in_the_mix(rmat22):
    """The serving workload at full size: the R-MAT scale-22 labels resident,
    labeling jobs of the batched workload's size distribution admitted
    beside them, 300 requests of 1..65,536 uniform pairs (seed 4) arriving
    while jobs build.  Every answer in the mix equals the same pairs answered
    alone; the answers from three sources equal BFS distances."""
    from paper_1906_12018_gb300.serve import LabelServer

    g, order, lab = rmat22
    srv = LabelServer(build_slots=2, max_inflight=2)
    try:
        srv.add_resident("base", lab)
        for i in range(6):
            s = G.small_graph(i)
            srv.submit_build(f"job{i}", s.off, s.col, G.degree_order(s))
        rng = np.random.default_rng(4)
        reqs = [srv.submit_query("base", rng.integers(0, g.n, (int(rng.integers(1, 65537)), 2)).astype(np.int32))
                for _ in range(300)]
        srv.wait_idle()
        allp = np.concatenate([r.pairs for r in reqs])
        alone = gpu_query(lab, allp)
        assert np.array_equal(np.concatenate([r.result for r in reqs]), alone)
        srcs = rng.choice(g.n, 3, replace=False)
        for s in srcs:
            D = O.bfs(g.off, g.col, int(s))
            tg = rng.integers(0, g.n, 2000).astype(np.int32)
            pairs = np.stack([np.full(2000, s, np.int32), tg], 1)
            assert np.array_equal(gpu_query(lab, pairs), D[tg])
        assert len(srv.completed_builds) == 6
    finally:
        for nm in list(srv.sets):
            if nm != "base":
                srv.drop(nm)
        srv.sets.pop("base", None)
        srv.close()
