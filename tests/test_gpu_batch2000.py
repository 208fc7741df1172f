"""The batched workload at full size: 2,000 graphs (graph i: seed 100 + i,
n_i = round(2^U(10,16)); even i R-MAT edge factor 8 with its largest
component, odd i Chung-Lu exponent 2.3, mean degree 10), labeled by one
plb_build_batch call.  Every part's labels must equal the oracle's: the
stored SHA-256 of each graph's oracle labels (tests/golden/batch2000_labels.json,
written by tests/golden/make_digests.py from the oracle's PLL alone) against
the same digest of the GPU labels.  Checked with the batch API's defaults
(captured round loop) and with the tier geometry the autotuner picks."""
import json
import os
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1906_12018_gb300 import autotune  # noqa: E402
from paper_1906_12018_gb300 import graphs as G  # noqa: E402
from paper_1906_12018_gb300 import plb  # noqa: E402

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
sys.path.insert(0, GOLDEN)
import label_digest as LD  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def batch2000():
    with open(os.path.join(GOLDEN, "batch2000_labels.json")) as f:
        want = json.load(f)["graphs"]
    dev = torch.device("cuda:0")
    parts = []
    for i in range(len(want)):
        g = G.small_graph(i)
        o = G.degree_order(g)
        parts.append((torch.from_numpy(g.off).to(dev), torch.from_numpy(g.col).to(dev),
                      torch.from_numpy(o).to(dev)))
        assert (g.n, g.m) == (want[i]["n"], want[i]["m"]), i
    yield want, parts
    del parts
    torch.cuda.empty_cache()


def _check_all(labs, want):
    bad = []
    for i, (lab, w) in enumerate(zip(labs, want)):
        off, hub, dist = lab.to_host()
        if lab.total != w["labels"] or LD.labels_digest(off, hub, dist) != w["sha256"]:
            bad.append(i)
    return bad


def test_batch2000_default_options_equal_oracle(batch2000):
    want, parts = batch2000
    labs = plb.build_batch(parts)
    try:
        assert _check_all(labs, want) == []
    finally:
        for lab in labs:
            lab.free()


def test_batch2000_tuned_options_equal_oracle(batch2000, tmp_path, monkeypatch):
    want, parts = batch2000
    monkeypatch.setenv("PLB_AUTOTUNE_CACHE", str(tmp_path / "autotune.json"))
    tuned, _ = autotune.tune_batch(parts[:200], reps=1)
    labs = plb.build_batch(parts, tuned)
    try:
        assert _check_all(labs, want) == []
    finally:
        for lab in labs:
            lab.free()


def test_batch2000_sampled_queries_match_single_builds(batch2000):
    """A few parts answered from the batch equal the same graphs built alone."""
    want, parts = batch2000
    labs = plb.build_batch(parts)
    try:
        for i in (0, 1, 999, 1998, 1999):
            single = plb.build(*parts[i])
            n = want[i]["n"]
            pairs = torch.from_numpy(G.uniform_pairs(n, 2000, 11 + i)).cuda()
            a = labs[i].query(pairs)
            b = single.query(pairs)
            torch.cuda.synchronize()
            assert np.array_equal(a.cpu().numpy(), b.cpu().numpy()), i
            single.free()
    finally:
        for lab in labs:
            lab.free()
