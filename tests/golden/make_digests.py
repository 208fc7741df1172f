"""Write the stored label digests that the full-size GPU parity tests compare
against.  Calls only the oracle (``oracle/``) and the input generator.

    python tests/golden/make_digests.py rmat22     # -> tests/golden/rmat22_labels.json
    python tests/golden/make_digests.py batch [P]  # -> tests/golden/batch2000_labels.json

``rmat22``: R-MAT scale 22, edge factor 16, seed 3, largest component
(2,394,833 vertices), degree order; the oracle's sequential PLL (Alg. 1 with
the small revision) runs once on one core; the labels are digested per block
of 2^16 rows (``label_digest.block_digests``).  Its wall time is stored with
the host it ran on (the oracle's full-run time for this workload).

``batch``: the 2,000 graphs of the batched workload (graph i: seed 100 + i,
n_i = round(2^U(10,16)); even i R-MAT edge factor 8 with its largest
component, odd i Chung-Lu exponent 2.3, mean degree 10), each labeled by the
same PLL in its own degree order and digested whole.  The graphs run as
independent jobs over P processes (default: all cores; spawn-started); each
job's single-core time and the pool's wall time are stored too.
"""
import json
import multiprocessing as mp
import os
import platform
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
for p in (ROOT, HERE):
    if p not in sys.path:
        sys.path.insert(0, p)

import label_digest as LD  # noqa: E402

N_BATCH = 2000


def _host():
    cpu = ""
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith(("model name", "cpu part")):
                    cpu = line.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    return {"machine": platform.machine(), "cpu": cpu, "nproc": os.cpu_count()}


def make_rmat22():
    import oracle as O
    from paper_1906_12018_gb300 import graphs as G

    g = G.workload("rmat22")
    order = G.degree_order(g)
    t = time.perf_counter()
    lab = O.pll(g.off, g.col, order)
    el = time.perf_counter() - t
    digests = LD.block_digests(lab.off, lab.hub, lab.dist)
    rec = {"workload": "rmat22", "n": g.n, "m": g.m, "labels": lab.total, "max_dist": lab.max_dist,
           "block_rows": LD.BLOCK_ROWS, "blocks": digests, "pll_seconds": round(el, 1),
           "host": _host()}
    with open(os.path.join(HERE, "rmat22_labels.json"), "w") as f:
        json.dump(rec, f, indent=1)
    print({k: v for k, v in rec.items() if k != "blocks"}, flush=True)


def _batch_job(i):
    import oracle as O
    from paper_1906_12018_gb300 import graphs as G

    g = G.small_graph(i)
    order = G.degree_order(g)
    t = time.perf_counter()
    lab = O.pll(g.off, g.col, order)
    el = time.perf_counter() - t
    return i, g.n, g.m, lab.total, LD.labels_digest(lab.off, lab.hub, lab.dist), el


def make_batch(procs):
    t = time.perf_counter()
    rows = [None] * N_BATCH
    with mp.get_context("spawn").Pool(procs) as pool:
        for i, n, m, total, dig, el in pool.imap_unordered(_batch_job, range(N_BATCH), chunksize=4):
            rows[i] = {"n": n, "m": m, "labels": total, "sha256": dig, "pll_seconds": round(el, 4)}
    wall = time.perf_counter() - t
    rec = {"workload": "batch2000", "graphs": rows, "pll_seconds_one_core_sum": round(sum(r["pll_seconds"] for r in rows), 2),
           "pool_wall_seconds": round(wall, 2), "pool_processes": procs, "host": _host()}
    with open(os.path.join(HERE, "batch2000_labels.json"), "w") as f:
        json.dump(rec, f, indent=0)
    print({k: v for k, v in rec.items() if k != "graphs"}, flush=True)


if __name__ == "__main__":
    what = sys.argv[1] if len(sys.argv) > 1 else ""
    if what == "rmat22":
        make_rmat22()
    elif what == "batch":
        make_batch(int(sys.argv[2]) if len(sys.argv) > 2 else (os.cpu_count() or 1))
    else:
        sys.exit(__doc__)
