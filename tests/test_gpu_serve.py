"""Serving: labeling jobs and query requests submitted together; every query
answer equals the answer of the same request run alone, and every built label
set equals a build run alone (integers: tolerance 0)."""
import numpy as np
import pytest
import torch

from paper_1906_12018_gb300 import graphs as G
from paper_1906_12018_gb300 import plb
from paper_1906_12018_gb300.serve import LabelServer, latency_summary

import oracle as O  # noqa: E402
from gpu_util import gpu_build, gpu_query, host_labels

pytestmark = pytest.mark.gpu


def test_results_identical_alone_and_in_the_mix():
    base = G.workload("rmat12")
    base_order = G.degree_order(base)
    jobs = [G.small_graph(i) for i in (3, 5, 8, 13)]
    srv = LabelServer(build_slots=2, max_inflight=2, max_pairs_per_launch=20_000)
    try:
        srv.add_resident("base", gpu_build(base, base_order))
        futs = {f"job{i}": srv.submit_build(f"job{i}", g.off, g.col, G.degree_order(g)) for i, g in enumerate(jobs)}
        rng = np.random.default_rng(9)
        reqs = []
        for k in range(60):
            name = "base" if k % 3 else f"job{k % 4}"
            n = base.n if name == "base" else jobs[int(name[3:])].n
            q = int(rng.integers(1, 6000))
            reqs.append((name, srv.submit_query(name, rng.integers(0, n, (q, 2)).astype(np.int32))))
        srv.wait_idle()
        built = {nm: f.result() for nm, f in futs.items()}
        # labels identical to a build alone
        for i, g in enumerate(jobs):
            alone = host_labels(gpu_build(g, G.degree_order(g)))
            mixed = host_labels(built[f"job{i}"])
            for a, b in zip(alone, mixed):
                assert np.array_equal(a, b)
        # every request identical to the same pairs queried alone
        for name, r in reqs:
            lab = srv.sets[name]
            assert np.array_equal(r.result, gpu_query(lab, r.pairs)), name
        # and a sample of the mixed answers equals BFS distances
        for name, r in [x for x in reqs if x[0] == "base"][:4]:
            for s in np.unique(r.pairs[:, 0])[:5]:
                D = O.bfs(base.off, base.col, int(s))
                m = r.pairs[:, 0] == s
                assert np.array_equal(r.result[m], D[r.pairs[m, 1]])
        st = latency_summary([r for _, r in reqs])
        assert st["requests"] == 60 and st["p99_ms"] >= st["p50_ms"] > 0
    finally:
        srv.close()


def test_autotuned_options_keep_labels_identical(tmp_path, monkeypatch):
    from paper_1906_12018_gb300 import autotune

    monkeypatch.setenv("PLB_AUTOTUNE_CACHE", str(tmp_path / "tune.json"))
    gs = [G.small_graph(i) for i in range(6)]
    devs = []
    for g in gs:
        rp = torch.from_numpy(g.off).cuda()
        devs.append((rp, torch.from_numpy(g.col).cuda(), torch.from_numpy(G.degree_order(g)).cuda()))
    opts, rep = autotune.tune_batch(devs, space={"warp_cand_cap": [256, 1024], "block_threads": [256]}, reps=1)
    assert not rep["cached"] and rep["trials"] >= 2
    opts2, rep2 = autotune.tune_batch(devs, space={"warp_cand_cap": [256, 1024], "block_threads": [256]})
    assert rep2["cached"] and autotune.as_dict(opts2) == autotune.as_dict(opts)
    tuned = plb.build_batch(devs, opts)
    plain = plb.build_batch(devs)
    for a, b in zip(tuned, plain):
        for x, y in zip(host_labels(a), host_labels(b)):
            assert np.array_equal(x, y)


def test_admission_under_a_small_hbm_budget():
    """A budget that holds about two build footprints beside the resident
    set: jobs wait for memory, the admitted footprints never exceed the
    budget, every job completes, and its labels equal a build run alone."""
    from paper_1906_12018_gb300.serve import build_footprint

    base = G.workload("rmat12")
    jobs = [G.small_graph(i) for i in range(8)]
    fps = [build_footprint(g.n, g.nnz) for g in jobs]
    resident = gpu_build(base, G.degree_order(base))
    budget = resident.nbytes() + int(2.2 * max(fps))
    srv = LabelServer(hbm_budget=budget, build_slots=4, max_inflight=2)
    try:
        srv.add_resident("base", resident)
        futs = [srv.submit_build(f"job{i}", g.off, g.col, G.degree_order(g)) for i, g in enumerate(jobs)]
        srv.wait_idle()
        assert srv.peak_used <= budget
        for i, (g, f) in enumerate(zip(jobs, futs)):
            alone = host_labels(gpu_build(g, G.degree_order(g)))
            for a, b in zip(alone, host_labels(f.result())):
                assert np.array_equal(a, b), i
    finally:
        srv.close()
