"""Write oracle/workload_totals.json: per named workload, the vertex and edge
counts and the canonical label total / largest distance computed by the
oracle's sequential PLL (Alg. 1), with its single-thread wall time.  A name
``w:<workload>`` is that graph with per-edge weights uniform on 1..7 (seed 2)
labeled by the oracle's PLL with pruned Dijkstra searches.

The benchmark's CPU-baseline leg times a bounded prefix of the same PLL run
and scales it to the whole workload by the share of these labels it produced.

    python oracle/workload_totals.py chunglu20 rmat12 w:chunglu20
"""
import json
import os
import platform
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402
from paper_1906_12018_gb300 import graphs as G  # noqa: E402

PATH = os.path.join(HERE, "workload_totals.json")


def main(names):
    data = {}
    if os.path.exists(PATH):
        with open(PATH) as f:
            data = json.load(f)
    for name in names:
        weighted = name.startswith("w:")
        g = G.workload(name[2:] if weighted else name)
        order = G.degree_order(g)
        t = time.perf_counter()
        if weighted:
            lab = O.pll_weighted(g.off, g.col, G.edge_weights(g, 1, 7, 2), order)
        else:
            lab = O.pll(g.off, g.col, order)
        el = time.perf_counter() - t
        data[name] = {"n": g.n, "m": g.m, "labels": lab.total, "max_dist": lab.max_dist,
                      "pll_seconds": round(el, 2), "machine": platform.machine()}
        print(name, data[name], flush=True)
    with open(PATH, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)


if __name__ == "__main__":
    main(sys.argv[1:] or ["rmat12", "chunglu20"])
