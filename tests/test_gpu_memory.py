"""Device memory of a build, read from the library's pool (plb_memory_stats):
the high mark covers the label set, memory returns to the pool when the set
is freed, and the admission footprint of the serving loop
(serve.build_footprint) is at least the measured peak on graphs of several
sizes and shapes."""
import pytest

from gpu_util import build_peak
from paper_1906_12018_gb300 import graphs as G
from paper_1906_12018_gb300.serve import build_footprint

pytestmark = pytest.mark.gpu


def test_memory_stats_follow_a_build():
    m = build_peak(G.workload("rmat12"))
    assert m["labels"] > 0
    assert m["kept"] >= m["labels"]  # the label set's rows come from the pool
    assert m["peak"] >= m["kept"]
    assert m["left"] == 0  # freeing the set returns its blocks to the pool


@pytest.mark.parametrize("name", ["small3", "small8", "rmat12", "rmat16-16-5", "chunglu131072-16-2.1-7",
                                  "chunglu20"])
def test_build_footprint_covers_the_measured_peak(name):
    g = G.small_graph(int(name[5:])) if name.startswith("small") else G.workload(name)
    m = build_peak(g)
    assert 0 < m["peak"] <= build_footprint(g.n, g.nnz) - m["inputs"], (m, build_footprint(g.n, g.nnz))
