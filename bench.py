#!/usr/bin/env python3
"""Labeling throughput benchmark (edges/sec, % of HBM roofline) plus batched
query throughput/latency, on synthetic power-law graphs.

Default workload: R-MAT scale 22 (edge factor 16, (a,b,c,d) =
(0.57,0.19,0.19,0.05), seed 3, largest component: 2,394,833 vertices,
64,152,981 edges), degree-descending order (ties by id).  One step = one
plb_build of the whole graph (all rounds, from the rank-space relabel to the
final by-id label layout) with the CSR already resident on the device.  The
same line carries sub-objects for the Chung-Lu 2^20 build, the batched
workload (2,000 small graphs) and the serving loop with the R-MAT labels
resident.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

With N > 1 (torchrun, one rank per GPU) every rank labels its own replica of
the graph (a single graph is not partitioned); value = edges of all ranks /
max-over-ranks time ("replicas", weak scaling).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def algorithmic_bytes(st: dict, n: int) -> dict:
    """Bytes the method itself must move in one build, by the cost terms of
    Sec. 3.3 / 4.3, from the build's own exact counters:

    * csr:   8 per receiver-round (its CSR row bounds) + 4 per arc scanned
             (the edge-access term, O(D|E|));
    * cand:  4 per message (a frontier hub h < v read before dedup; the
             distance is implicit in the round);
    * check: 5 per label entry the distance checks read.  "check" counts
             the entries the checks probe (each candidate scans the shorter
             side and stops at its first witness; candidates settled by the
             top-hub bitmasks probe none).  The paper's cost model (Sec. 4.3)
             scans, for every checked candidate, the entries of L(v) with
             hub < h ("check_lower", the side the paper scans) and, as an
             upper bound, also all of L(h) ("check_upper", the side it
             hashes); most of those reads are never made here, so a rate
             computed on them would exceed the HBM peak;
    * out:   5 per final label + 8 (n + 1) (the label CSR written once);
    * merge: 5 per label entry rewritten by the per-round merge (every row is
             rewritten in each round that accepts labels).
    The gather + prune kernels move csr + cand + check; out and merge belong
    to the finalise and merge kernels."""
    recv = sum(st["receivers"])
    csr = 8 * recv + 4 * st["arcs_scanned"]
    cand = 4 * st["messages"]
    chk = 5 * st["probed_entries"]
    chk_lo = 5 * st["check_lv_entries"]
    chk_hi = chk_lo + 5 * st["check_lh_entries"]
    out = 5 * st["total_labels"] + 8 * (n + 1)
    t, merge = n, 0
    for acc in st["accepted"]:
        if acc > 0:
            t += acc
            merge += 5 * t
    return {"csr": csr, "cand": cand, "check": chk, "check_lower": chk_lo, "check_upper": chk_hi, "out": out,
            "merge": merge, "gather_prune": csr + cand + chk, "gather_prune_cost_model_lower": csr + cand + chk_lo,
            "gather_prune_cost_model_upper": csr + cand + chk_hi}


# DRAM traffic of the gather + prune kernels, from ncu captures summarised in
# profiles/traffic.json, keyed by workload (valid only while the kernel
# sources hash to the recorded value).
TRAFFIC_RECORD = os.path.join(ROOT, "profiles", "traffic.json")
KERNEL_SOURCES = ("paper_1906_12018_gb300/csrc/plb_gather.cu", "paper_1906_12018_gb300/csrc/plb_kernels.cuh",
                  "paper_1906_12018_gb300/csrc/plb_internal.cuh")
# the round-1 kernels (k_round1_count, k_round1): their section of plb_round.cu
ROUND1_SECTION = ("paper_1906_12018_gb300/csrc/plb_round.cu", "// Both passes run flat over tiles of arcs",
                  "// Reset before re-running the gather/prune")


def round1_section() -> str:
    """Source of the round-1 kernels and of the file-local helpers ahead of
    them (the whole file when a marker is gone)."""
    rel, a, b = ROUND1_SECTION
    with open(os.path.join(ROOT, rel)) as f:
        text = f.read()
    i, j, k = text.find(a), text.find(b), text.find("}  // namespace")
    return text[:k] + text[i:j] if 0 <= k < i < j else text


def kernel_source_hash() -> str:
    """SHA-256 over the sources of the gather + prune class: the gather
    kernels' files and the round-1 kernels' section."""
    import hashlib

    h = hashlib.sha256()
    for rel in KERNEL_SOURCES:
        with open(os.path.join(ROOT, rel), "rb") as f:
            h.update(f.read())
    h.update(round1_section().encode())
    return h.hexdigest()


def recorded_traffic(workload: str):
    """The ncu record of this workload's gather + prune launches (DRAM bytes
    per launch and the capture it came from), or None when there is none or
    the kernels changed since."""
    try:
        with open(TRAFFIC_RECORD) as f:
            rec = json.load(f).get(workload)
    except (OSError, ValueError):
        return None
    if not rec or rec.get("kernel_sources_sha256") != kernel_source_hash():
        return None
    return rec


def measured_peaks() -> tuple[float, str]:
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks/throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.proc = None
        self.path = None

    def __enter__(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if self.proc is None or not self.path:
            return None
        rows = []
        with open(self.path) as f:
            for line in f:
                t = [x.strip() for x in line.split(",")]
                if len(t) >= 9:
                    rows.append(t)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def dist_init():
    import torch

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist

        dist.barrier()


def max_over_ranks(x: float, world: int) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist

    dev = "cpu" if dist.get_backend() == "gloo" else "cuda"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: float, ms_max: float, world: int) -> float:
    """Units per second of the whole job: every rank processes the same
    workload (replicas), timed by the slowest rank."""
    return units_per_rank * world / (ms_max / 1e3)


def host_cpu() -> dict:
    """The host the CPU baselines ran on: architecture, logical cores and CPU
    model (lscpu, else /proc/cpuinfo)."""
    import platform

    model = ""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    if not model:
        try:
            with open("/proc/cpuinfo") as f:
                for line in f:
                    if line.lower().startswith(("model name", "cpu part", "hardware")):
                        model = line.split(":", 1)[1].strip()
                        break
        except OSError:
            pass
    return {"machine": platform.machine(), "nproc": os.cpu_count(), "model": model}


def oracle_full_run(name: str) -> dict | None:
    """The record of a full oracle PLL run on a named workload: label total,
    single-core seconds and the host it ran on (oracle/workload_totals.py, or
    the stored digests of tests/golden/make_digests.py)."""
    try:
        with open(os.path.join(ROOT, "oracle", "workload_totals.json")) as f:
            rec = json.load(f).get(name)
        if rec:
            return {"labels": int(rec["labels"]), "seconds": rec.get("pll_seconds"),
                    "host": {"machine": rec.get("machine")}, "max_dist": rec.get("max_dist")}
    except (OSError, ValueError):
        pass
    try:
        with open(os.path.join(ROOT, "tests", "golden", f"{name}_labels.json")) as f:
            rec = json.load(f)
        return {"labels": int(rec["labels"]), "seconds": rec.get("pll_seconds"), "host": rec.get("host"),
                "max_dist": rec.get("max_dist")}
    except (OSError, ValueError, KeyError):
        return None


def oracle_total_labels(name: str) -> int | None:
    rec = oracle_full_run(name)
    return rec["labels"] if rec else None


def pll_sample(g, order, total: int, seconds: float) -> dict:
    """The oracle's sequential PLL (Alg. 1) on a bounded sample of this
    workload: the first roots in rank order for about `seconds`, scaled to the
    whole graph by the share of all labels produced (the total comes from a
    full oracle run).  Early roots produce labels fastest, so this estimate
    favours the CPU; both CPU legs of the benchmark use it with the same
    budget."""
    import oracle as O

    lab, roots, el = O.pll_budget(g.off, g.col, order, seconds)
    frac = lab.total / max(total, 1)
    est = el / max(frac, 1e-12)
    return {"value": g.m / est, "unit": "edges/s", "cores": 1, "kind": "oracle", "host": host_cpu(),
            "method": "prefix sample scaled by label share (an estimate that favours the CPU)",
            "sample": (f"PLL (Alg. 1) over the first {roots} roots in rank order ({el:.1f} s, "
                       f"{lab.total} of {total} labels = {100 * frac:.1f}%); time scaled by label share"),
            "sample_seconds": el}


def pll_full(g, order) -> dict:
    """The oracle's sequential PLL (Alg. 1) over the whole workload on one
    host core: its wall time, not an estimate."""
    import oracle as O

    t = time.perf_counter()
    lab = O.pll(g.off, g.col, order)
    el = time.perf_counter() - t
    return {"value": g.m / el, "unit": "edges/s", "cores": 1, "kind": "oracle", "host": host_cpu(),
            "method": "full run", "sample": f"PLL (Alg. 1) over all {g.n} roots ({lab.total} labels, {el:.1f} s)",
            "seconds": el}


def run_reference(args):
    """Reference arm: the CPU oracle on this workload (rank 0 only), timed the
    same way as the main line's cpu_baseline leg (a prefix sample of
    --cpu-seconds per timed step; warm-up steps take a 1 s sample)."""
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if rank != 0:
        return 0
    from paper_1906_12018_gb300 import graphs as G

    g = G.workload(args.workload)
    order = G.degree_order(g)
    total = oracle_total_labels(args.workload)
    if total is None:
        import oracle as O

        total = O.pll(g.off, g.col, order).total
    samples = []
    for step in range(args.warmup + args.steps):
        s = pll_sample(g, order, total, args.cpu_seconds if step >= args.warmup else 1.0)
        if step >= args.warmup:
            samples.append(s)
    v = statistics.median(s["value"] for s in samples)
    sec = statistics.median(s["sample_seconds"] for s in samples)
    full = oracle_full_run(args.workload)
    config = workload_config(args.workload, g, total)
    if full and full.get("max_dist") is not None:  # the same keys as the main line's config
        config = dict(config, rounds=int(full["max_dist"]) + 1,
                      parallelism="replicas" if world > 1 else "single", batch_hubs=args.batch_hubs)
    line = {"metric": "labeling edges/sec", "value": v, "unit": "edges/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1000 * sec, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "ms_per_step_is": "the timed oracle sample of one step (a prefix of the build), not a whole build",
            "estimated_ms_per_build": 1000 * g.m / v if v else None,
            "config": config, "impl": "reference",
            "cpu_baseline": {"kind": "oracle", "cores": 1, "value": v, "unit": "edges/s", "host": host_cpu(),
                             "method": samples[0]["method"], "sample": samples[0]["sample"]},
            "e2e": {"value": v, "unit": "edges/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    if full and full.get("seconds"):
        line["cpu_full_run"] = dict(full, value=g.m / float(full["seconds"]), unit="edges/s")
    print(json.dumps(line), flush=True)
    return 0


def workload_config(name: str, g, labels) -> dict:
    return {"workload": name, "n": g.n, "m": g.m, "labels": labels, "l2": "flushed between steps (256 MB write)"}


def _oracle_small_graph(i: int):
    """Worker: the oracle's PLL (Alg. 1) on graph i of the batched workload;
    (edges, labels, seconds of the labeling alone)."""
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    import oracle as O
    from paper_1906_12018_gb300 import graphs as G

    g = G.small_graph(i)
    order = G.degree_order(g)
    t = time.perf_counter()
    lab = O.pll(g.off, g.col, order)
    return g.m, lab.total, time.perf_counter() - t


def oracle_batch_sample(seconds: float, cores: int, limit: int = 2000) -> dict:
    """The oracle on a bounded sample of the batched workload: graphs 0, 1, ...
    labeled one after another on one core until `seconds` have passed, then
    the same graphs as independent jobs over `cores` processes (started with
    spawn: the caller may hold a CUDA context).  Edges per second of each."""
    import multiprocessing as mproc

    done, edges, t1 = 0, 0, 0.0
    while done < limit and t1 < seconds:
        m, _, el = _oracle_small_graph(done)
        edges += m
        t1 += el
        done += 1
    with mproc.get_context("spawn").Pool(cores) as pool:
        pool.map(_oracle_small_graph, range(min(cores, done)))  # start the workers
        t = time.perf_counter()
        pool.map(_oracle_small_graph, range(done), chunksize=1)
        tall = time.perf_counter() - t
    return {"value": edges / t1, "unit": "edges/s", "cores": 1, "kind": "oracle", "host": host_cpu(),
            "sample": f"PLL (Alg. 1) on graphs 0..{done - 1} of the batch ({edges} edges, {t1:.1f} s on one core)",
            "all_cores": {"value": edges / tall, "unit": "edges/s", "cores": cores,
                          "sample": f"the same {done} graphs as independent jobs ({tall:.1f} s wall, graph "
                                    "generation inside the jobs)"}}


def batch_report(args, steps: int, warmup: int, cpu: bool) -> dict:
    """2,000 small graphs (sizes log-uniform 1k-64k; half R-MAT edge factor 8,
    half Chung-Lu gamma 2.3 mean degree 10; seeds 100-2099): one plb_build
    per graph vs plb_build_batch over all of them (the batch API's defaults,
    a captured round loop, and the autotuned tier geometry).  The tuned
    batch's labels are compared, graph by graph, with the stored SHA-256 of
    the oracle's labels (tests/golden/batch2000_labels.json)."""
    import torch

    from paper_1906_12018_gb300 import autotune
    from paper_1906_12018_gb300 import graphs as G
    from paper_1906_12018_gb300 import plb

    dev = torch.device("cuda", 0)
    k = args.batch_graphs
    gs = [G.small_graph(i) for i in range(k)]
    devs = [(torch.from_numpy(g.off).to(dev), torch.from_numpy(g.col).to(dev),
             torch.from_numpy(G.degree_order(g)).to(dev)) for g in gs]
    m = sum(g.m for g in gs)
    opts = plb.default_options()
    tuned, tune_report = autotune.tune_batch(devs[: min(k, 200)])

    def timed(fn):
        torch.cuda.synchronize(dev)
        t = time.perf_counter()
        fn()
        torch.cuda.synchronize(dev)
        return time.perf_counter() - t

    def loop():
        for d in devs:
            plb.build(*d, opts).free()

    def batch(o):
        def f():
            for lab in plb.build_batch(devs, o):
                lab.free()
        return f

    for _ in range(max(warmup, 1)):
        timed(batch(None))
    t_loop = min(timed(loop) for _ in range(2))
    t_def = min(timed(batch(None)) for _ in range(max(steps, 1)))  # the batch API's defaults
    t_tuned = min(timed(batch(tuned)) for _ in range(max(steps, 1)))
    # the library pool's high mark over one tuned batched build
    torch.cuda.synchronize()
    mem0 = plb.memory_stats(reset=True)
    timed(batch(tuned))
    peak = plb.memory_stats()["used_high"] - mem0["used"]
    rep = {"workload": f"batch{k}", "graphs": k, "n": sum(g.n for g in gs), "m": m,
           "value": m / t_tuned, "unit": "edges/s", "ms": 1e3 * t_tuned,
           "one_graph_at_a_time": {"value": m / t_loop, "ms": 1e3 * t_loop},
           "batched_default": {"value": m / t_def, "ms": 1e3 * t_def, "use_graph": 1},
           "batched_tuned": {"value": m / t_tuned, "ms": 1e3 * t_tuned, "options": autotune.as_dict(tuned)},
           "speedup_vs_one_at_a_time": t_loop / t_tuned, "autotune": tune_report,
           "build_peak_bytes": peak}
    gold = os.path.join(ROOT, "tests", "golden", "batch2000_labels.json")
    if not args.no_parity_check and k == 2000 and os.path.exists(gold):
        sys.path.insert(0, os.path.dirname(gold))
        import label_digest as LD

        with open(gold) as f:
            want = json.load(f)
        labs = plb.build_batch(devs, tuned)
        bad = 0
        for lab, w in zip(labs, want["graphs"]):
            off, hub, dist = lab.to_host()
            bad += int(LD.labels_digest(off, hub, dist) != w["sha256"])
            lab.free()
        rep["parity"] = {"graphs": k, "equal_to_oracle": k - bad, "method": "SHA-256 per graph of the labels "
                         "(tuned options) against the oracle's, tests/golden/batch2000_labels.json"}
        rep["oracle_full_run"] = {"one_core_seconds_sum": want["pll_seconds_one_core_sum"],
                                  "pool_wall_seconds": want["pool_wall_seconds"],
                                  "pool_processes": want["pool_processes"], "host": want["host"],
                                  "value_one_core": m / want["pll_seconds_one_core_sum"],
                                  "value_pool": m / want["pool_wall_seconds"], "unit": "edges/s"}
    if cpu:
        rep["cpu_baseline"] = oracle_batch_sample(args.cpu_seconds, os.cpu_count() or 1, k)
    return rep


def run_batch(args):
    rep = batch_report(args, args.steps, args.warmup, not args.no_cpu_baseline)
    line = {"metric": "labeling edges/sec", "value": rep["value"], "unit": "edges/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": rep["ms"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": {"workload": rep["workload"], "graphs": rep["graphs"], "n": rep["n"], "m": rep["m"]},
            "cpu_baseline": rep.pop("cpu_baseline", None), "batch": rep}
    print(json.dumps(line), flush=True)
    return 0


def run_weighted(args):
    """Weighted labeling (Sec. 5.1; the weighted inputs of Sec. 6.1 draw each
    edge's weight uniformly from 1..7): the named workload with weights 1..7
    (seed 2); one step = one plb_build_weighted with the CSR and the weights
    resident on the device."""
    import torch

    from paper_1906_12018_gb300 import graphs as G
    from paper_1906_12018_gb300 import plb

    dev = torch.device("cuda", 0)
    g = G.workload(args.workload)
    wt = G.edge_weights(g, 1, 7, 2)
    order = G.degree_order(g)
    rp = torch.from_numpy(g.off).to(dev)
    col = torch.from_numpy(g.col).to(dev)
    w = torch.from_numpy(wt).to(dev)
    o = torch.from_numpy(order).to(dev)
    stream = torch.cuda.current_stream(dev)
    for _ in range(max(args.warmup, 3)):
        plb.build_weighted(rp, col, w, o).free()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    labs = []
    torch.cuda.synchronize(dev)
    with ClockSampler(0) as clk:
        for k in range(args.steps):
            flush.zero_()
            ev[k][0].record(stream)
            labs.append(plb.build_weighted(rp, col, w, o))
            ev[k][1].record(stream)
        torch.cuda.synchronize(dev)
    step_ms = [a.elapsed_time(b) for a, b in ev]
    ms = sum(step_ms) / len(step_ms)
    st0 = labs[0].stats()
    n_labels = labs[0].total
    launches = st0["launches"] * args.steps
    for lab in labs:
        lab.free()

    lab = plb.build_weighted(rp, col, w, o, plb.default_options(profile=1))
    st = lab.stats()
    gp_ms = sum(st["ms_gather_prune"])
    ab = algorithmic_bytes(st, g.n)
    gp_bytes = ab["gather_prune"]
    gp_launches = 2 * sum(1 for r in st["receivers"] if r > 0)  # warp tier + block tier per round with receivers
    peak, peak_kind = measured_peaks()
    achieved = gp_bytes / (gp_ms / 1e3) / 1e9 if gp_ms > 0 else 0.0
    qpairs = torch.from_numpy(G.uniform_pairs(g.n, 1 << 16, 4)).to(dev)
    out = torch.empty(1 << 16, dtype=torch.int32, device=dev)
    for _ in range(3):
        lab.query(qpairs, out)
    qev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(20)]
    for a, b in qev:
        flush.zero_()
        a.record(stream)
        lab.query(qpairs, out)
        b.record(stream)
    torch.cuda.synchronize(dev)
    qms = statistics.median(a.elapsed_time(b) for a, b in qev)
    lab.free()

    # end to end: pinned host CSR, weights and order -> device, build, labels -> pinned host
    h_in = [torch.from_numpy(x).pin_memory() for x in (g.off, g.col, wt, order)]
    h2d = sum(t.numel() * t.element_size() for t in h_in)
    h_off = torch.empty(g.n + 1, dtype=torch.int64, pin_memory=True)
    h_hub = torch.empty(n_labels, dtype=torch.int32, pin_memory=True)
    h_dist = torch.empty(n_labels, dtype=torch.uint8, pin_memory=True)
    d2h = h_off.numel() * 8 + h_hub.numel() * 4 + h_dist.numel()
    e2e_ms = []
    for k in range(args.e2e_steps + 1):
        flush.zero_()
        torch.cuda.synchronize(dev)
        t = time.perf_counter()
        d_rp, d_col, d_w, d_o = (x.to(dev, non_blocking=True) for x in h_in)
        lab = plb.build_weighted(d_rp, d_col, d_w, d_o)
        off_d, hub_d, dist_d = lab.device_arrays()
        h_off.copy_(off_d, non_blocking=True)
        h_hub.copy_(hub_d, non_blocking=True)
        h_dist.copy_(dist_d, non_blocking=True)
        torch.cuda.synchronize(dev)
        if k > 0:
            e2e_ms.append(1e3 * (time.perf_counter() - t))
        lab.free()
    e2e_med = statistics.median(e2e_ms)

    cpu = None
    total = oracle_total_labels("w:" + args.workload)
    if not args.no_cpu_baseline and total is not None:
        import oracle as O

        part, roots, el = O.pll_weighted_budget(g.off, g.col, wt, order, args.cpu_seconds)
        frac = part.total / max(total, 1)
        cpu = {"value": g.m / (el / max(frac, 1e-12)), "unit": "edges/s", "cores": 1, "kind": "oracle",
               "host": host_cpu(),
               "sample": (f"PLL with pruned Dijkstra searches over the first {roots} roots in rank order "
                          f"({el:.1f} s, {part.total} of {total} labels = {100 * frac:.1f}%); time scaled by "
                          "label share")}
    line = {"metric": "labeling edges/sec (weighted)", "value": g.m / (ms / 1e3), "unit": "edges/s", "n_gpus": 1,
            "steps": args.steps, "warmup": max(args.warmup, 3), "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": {"workload": f"{args.workload} weights 1..7 (seed 2)", "n": g.n, "m": g.m,
                       "labels": n_labels, "rounds": st0["rounds"], "max_dist": int(max(  # the per-round lists start at round 1
                           (d + 1 for d, a in enumerate(st0["accepted"]) if a > 0), default=0)),
                       "l2": "flushed between steps (256 MB write)"},
            "roofline": {"bound": "hbm", "kernel": "gather+prune (k_gp_warp, k_gp_block)", "achieved": achieved,
                         "peak": peak, "unit": "GB/s", "frac": achieved / peak if peak else None,
                         "peak_kind": peak_kind, "traffic": None, "algorithmic_bytes": gp_bytes,
                         "bytes_by_term": ab, "launches_per_build": gp_launches, "kernel_ms": gp_ms},
            "kernel_ms": {"prepare": st["ms_prepare"], "frontier": st["ms_frontier"],
                          "gather_prune": st["ms_gather_prune"][0], "merge_sort_index": st["ms_merge"],
                          "finalize": st["ms_finalize"]},
            "e2e": {"value": g.m / (e2e_med / 1e3), "unit": "edges/s", "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h, "ms_per_step": e2e_med},
            "queries": {"value": (1 << 16) / (qms / 1e3), "unit": "queries/s", "batch": 1 << 16},
            "gpu_launches": launches, "clocks": clk.summary(), "cpu_baseline": cpu}
    print(json.dumps(line), flush=True)
    return 0


def run_directed(args):
    """Directed labeling (Sec. 5.1): R-MAT arcs kept directed (2^scale vertices,
    edge factor 16, seed 3), in + out degree order; one step = one
    plb_build_directed (L_in and L_out) with the arcs resident on the device."""
    import torch

    from paper_1906_12018_gb300 import graphs as G
    from paper_1906_12018_gb300 import plb

    dev = torch.device("cuda", 0)
    g = G.rmat_digraph(args.directed_scale, 16, 3)
    order = G.directed_degree_order(g)
    rp = torch.from_numpy(g.off).to(dev)
    col = torch.from_numpy(g.col).to(dev)
    o = torch.from_numpy(order).to(dev)
    stream = torch.cuda.current_stream(dev)
    for _ in range(max(args.warmup, 3)):
        for lab in plb.build_directed(rp, col, o):
            lab.free()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    labs = None
    for k in range(args.steps):
        flush.zero_()
        ev[k][0].record(stream)
        labs = plb.build_directed(rp, col, o)
        ev[k][1].record(stream)
        torch.cuda.synchronize(dev)
        if k + 1 < args.steps:
            for lab in labs:
                lab.free()
    ms = statistics.median(a.elapsed_time(b) for a, b in ev)
    lin, lout = labs
    st_in, st_out = lin.stats(), lout.stats()
    pairs = torch.from_numpy(G.uniform_pairs(g.n, 1 << 16, 4)).to(dev)
    out = torch.empty(1 << 16, dtype=torch.int32, device=dev)
    for _ in range(3):
        plb.query_directed(lout, lin, pairs, out)
    qev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(20)]
    for a, b in qev:
        flush.zero_()
        a.record(stream)
        plb.query_directed(lout, lin, pairs, out)
        b.record(stream)
    torch.cuda.synchronize(dev)
    qms = statistics.median(a.elapsed_time(b) for a, b in qev)
    line = {"metric": "labeling arcs/sec (directed)", "value": g.arcs / (ms / 1e3), "unit": "arcs/s", "n_gpus": 1,
            "steps": args.steps, "warmup": max(args.warmup, 3), "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": {"workload": f"rmat-directed{args.directed_scale}-16-3", "n": g.n, "arcs": g.arcs,
                       "labels_in": lin.total, "labels_out": lout.total, "rounds": [st_in["rounds"], st_out["rounds"]],
                       "l2": "flushed between steps (256 MB write)"},
            "queries": {"value": (1 << 16) / (qms / 1e3), "unit": "queries/s", "batch": 1 << 16},
            "gpu_launches": st_in["launches"] * args.steps}
    print(json.dumps(line), flush=True)
    lin.free()
    lout.free()
    return 0


def serve_report(args, base, g, rates, seconds: float) -> dict:
    """Serving with the label set `base` (of graph g) resident: labeling jobs
    drawn from the small-graph distribution, submitted every
    --serve-job-interval seconds and admitted by HBM footprint; query
    requests with Poisson arrivals and uniform 1..65,536 pairs (seed 4), at
    each offered load of `rates` for `seconds`.  Every request answered in
    the mix is compared with the same pairs answered alone."""
    import threading

    import torch

    from paper_1906_12018_gb300 import graphs as G
    from paper_1906_12018_gb300.serve import LabelServer, latency_summary

    dev = torch.device("cuda", 0)
    jobs = [G.small_graph(i) for i in range(args.serve_jobs)]

    def run_load(rate: float, check: bool) -> dict:
        srv = LabelServer(build_slots=2, max_inflight=2)
        srv.add_resident("base", base)
        stop = time.perf_counter() + seconds
        rng = np.random.default_rng(4)
        reqs = []

        def jobs_client():
            i = 0
            while time.perf_counter() < stop and i < len(jobs):
                gi = jobs[i]
                srv.submit_build(f"job{i}", gi.off, gi.col, G.degree_order(gi))
                i += 1
                time.sleep(args.serve_job_interval)

        jt = threading.Thread(target=jobs_client)
        jt.start()
        t0 = t_next = time.perf_counter()
        while time.perf_counter() < stop:
            t_next += rng.exponential(1.0 / rate)
            delay = t_next - time.perf_counter()
            if delay > 0:
                time.sleep(delay)
            q = int(rng.integers(1, 65537))
            reqs.append(srv.submit_query("base", rng.integers(0, g.n, (q, 2)).astype(np.int32)))
        jt.join()
        srv.wait_idle()
        st = latency_summary(reqs)
        st["offered_requests_per_s"] = rate
        st["achieved_requests_per_s"] = len(reqs) / max(max(r.t_done for r in reqs) - t0, 1e-9)
        st["jobs_done"] = len(srv.completed_builds)
        if check:  # every result in the mix = the same pairs answered alone
            allp = np.concatenate([r.pairs.reshape(-1, 2) for r in reqs]).astype(np.int32)
            alone = base.query(torch.from_numpy(allp).to(dev)).cpu().numpy()
            mixed = np.concatenate([r.result for r in reqs])
            st["identical_alone"] = {"requests": len(reqs), "pairs": int(allp.shape[0]),
                                     "equal": bool(np.array_equal(alone, mixed))}
        for nm in list(srv.sets):
            if nm != "base":
                srv.drop(nm)
        srv.sets.pop("base")
        srv.close()
        return st

    results = [run_load(rate, check=True) for rate in rates]
    # knee: the highest offered load the server keeps up with (requests
    # answered at >= 95% of the offered rate) while p99 stays within 4x the
    # lightest load's p99; then one more load at 70% of it
    p99_0 = results[0]["p99_ms"]
    fine = [r for r in results if r["achieved_requests_per_s"] >= 0.95 * r["offered_requests_per_s"]
            and r["p99_ms"] <= 4 * p99_0]
    knee = max(fine, key=lambda r: r["offered_requests_per_s"]) if fine else results[0]
    at70 = run_load(0.7 * knee["offered_requests_per_s"], check=True)
    return {"workload": f"serve-{args.serve_resident}", "n": g.n, "m": g.m, "labels": base.total,
            "value": knee["queries_per_s"], "unit": "queries/s", "p50_ms": knee["p50_ms"], "p99_ms": knee["p99_ms"],
            "request_pairs": "uniform 1..65536", "arrivals": "poisson", "seconds": seconds,
            "job_interval_s": args.serve_job_interval,
            "knee_rule": "highest offered load with >= 95% answered and p99 <= 4x the lightest load's",
            "latency": "arrival (submit) to distances on the host, per request",
            "knee": knee, "at_70pct_of_knee": at70, "loads": results}


def run_serve(args):
    """Serving: R-MAT scale-22 labels resident (see serve_report)."""
    import torch

    from paper_1906_12018_gb300 import graphs as G
    from paper_1906_12018_gb300 import plb

    dev = torch.device("cuda", 0)
    g = G.workload(args.serve_resident)
    order = G.degree_order(g)
    base = plb.build(torch.from_numpy(g.off).to(dev), torch.from_numpy(g.col).to(dev),
                     torch.from_numpy(order).to(dev))
    rep = serve_report(args, base, g, args.serve_rates, args.serve_seconds)
    line = {"metric": "queries/sec with p50/p99 latency", "value": rep["value"], "unit": "queries/s",
            "n_gpus": 1, "steps": len(rep["loads"]) + 1, "warmup": 0, "ms_per_step": None, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": {"workload": rep["workload"], "n": g.n, "m": g.m, "labels": base.total},
            "p50_ms": rep["p50_ms"], "p99_ms": rep["p99_ms"], "serving": rep}
    print(json.dumps(line), flush=True)
    base.free()
    return 0


def measure_build(args, g, order, dev, steps: int, warmup: int, e2e_steps: int, world: int = 1, local: int = 0):
    """One workload: `steps` timed plb_build calls with the CSR resident
    (CUDA events on the build's stream, L2 flushed between steps), a profiled
    build for the kernel-class times and counters (the roofline of the
    gather + prune class), batched queries, and the end-to-end build through
    the public API with host copies."""
    import torch

    from paper_1906_12018_gb300 import graphs as G
    from paper_1906_12018_gb300 import plb

    rp = torch.from_numpy(g.off).to(dev)
    col = torch.from_numpy(g.col).to(dev)
    o = torch.from_numpy(order).to(dev)
    stream = torch.cuda.current_stream(dev)
    opts = plb.default_options(batch_hubs=args.batch_hubs)
    for _ in range(warmup):
        lab = plb.build(rp, col, o, opts)
        lab.free()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)  # > 129 MB L2

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    torch.cuda.synchronize(dev)
    barrier(world)
    n_labels, st0 = None, None
    with ClockSampler(local if world > 1 else 0) as clk:
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        for k in range(steps):
            flush.zero_()  # L2 flush between steps (outside the events)
            ev[k][0].record(stream)
            lab = plb.build(rp, col, o, opts)
            ev[k][1].record(stream)
            if k == 0:
                n_labels, st0 = lab.total, lab.stats()
            lab.free()  # stream-ordered: the next build reuses the memory
        torch.cuda.synchronize(dev)
        wall = time.perf_counter() - t0
    barrier(world)
    step_ms = [a.elapsed_time(b) for a, b in ev]
    ms = sum(step_ms) / len(step_ms)
    ms_max = max_over_ranks(ms, world)
    launches = st0["launches"] * steps

    # kernel-class timings and counters: one profiled build; around it the
    # high mark of the library's memory pool (the build's device memory
    # beyond the caller's CSR, against the serving loop's footprint model)
    from paper_1906_12018_gb300.serve import build_footprint

    torch.cuda.synchronize(dev)
    mem0 = plb.memory_stats(reset=True)
    lab = plb.build(rp, col, o, plb.default_options(profile=1, batch_hubs=args.batch_hubs))
    st = lab.stats()
    torch.cuda.synchronize(dev)
    mem1 = plb.memory_stats()
    in_bytes = rp.numel() * 8 + col.numel() * 4 + o.numel() * 4
    memory = {"build_peak_bytes": mem1["used_high"] - mem0["used"], "labels_bytes": lab.nbytes(),
              "footprint_model_bytes": build_footprint(g.n, g.nnz) - in_bytes, "input_bytes": in_bytes}
    gp_ms = sum(st["ms_gather_prune"])
    ab = algorithmic_bytes(st, g.n)
    # round 1: k_round1_count and k_round1; every later host-driven round: the
    # block tier, the warp tier and the block tier over the warp tier's escalations
    gp_launches = 2 + 3 * (st["rounds"] - 1)
    traffic = recorded_traffic(args.workload)
    peak, peak_kind = measured_peaks()
    rate = (lambda b: b / (gp_ms / 1e3) / 1e9) if gp_ms > 0 else (lambda b: 0.0)
    achieved = rate(ab["gather_prune"])
    roof = {"bound": "hbm", "kernel": "gather+prune (k_round1_count, k_round1, k_gp_warp, k_gp_block)",
            "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak if peak else None,
            "peak_kind": peak_kind, "frac_vs_nominal_8tbs": achieved / 8000.0,
            "algorithmic_bytes_per_launch": ab["gather_prune"] / gp_launches,
            "launches_per_build": gp_launches, "kernel_ms": gp_ms, "bytes_by_term": ab,
            "bytes_rule": "csr + cand + check (entries probed); out and merge belong to other kernels",
            "cost_model_rates": {"lower": rate(ab["gather_prune_cost_model_lower"]),
                                 "upper": rate(ab["gather_prune_cost_model_upper"]), "unit": "GB/s",
                                 "note": "the paper's check reads (Sec. 4.3), mostly skipped here"},
            "traffic": None, "build_ms_profiled": st["ms_total"]}
    if traffic:
        roof["traffic"] = traffic["dram_bytes_per_launch"]
        roof["traffic_source"] = traffic["source"]
        roof["traffic_over_algorithmic"] = traffic["dram_bytes_per_launch"] / roof["algorithmic_bytes_per_launch"]
        hbm_ncu = traffic["dram_bytes_per_launch"] * gp_launches / (gp_ms / 1e3) / 1e9 if gp_ms > 0 else 0.0
        roof["hbm_frac_ncu"] = hbm_ncu / peak if peak else None

    # batched queries on the resident labels: 65,536 uniform pairs per launch
    qpairs = torch.from_numpy(G.uniform_pairs(g.n, 1 << 16, 4)).to(dev)
    out = torch.empty(1 << 16, dtype=torch.int32, device=dev)
    for _ in range(3):
        lab.query(qpairs, out)
    qev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(20)]
    for a, b in qev:
        flush.zero_()
        a.record(stream)
        lab.query(qpairs, out)
        b.record(stream)
    torch.cuda.synchronize(dev)
    qms = sorted(a.elapsed_time(b) for a, b in qev)
    q_value = (1 << 16) / (statistics.median(qms) / 1e3)
    q_bytes = None
    if st["total_labels"]:
        # per pair: 4 B x (|L(s)| + |L(t)|) of packed entries + 12 B of pair and answer
        off_d = lab.device_arrays()[0]
        rl = (off_d[1:] - off_d[:-1]).to(torch.int64)
        # pairs are by original id; row lengths are indexed by original id
        pr = qpairs.view(-1, 2).to(torch.int64)
        q_bytes = float((4 * (rl[pr[:, 0]] + rl[pr[:, 1]]) + 12).sum().item())
    lab.free()
    qroof = {"bound": "hbm", "achieved": (q_bytes / (statistics.median(qms) / 1e3) / 1e9) if q_bytes else None,
             "peak": peak, "unit": "GB/s"}
    if q_bytes:
        qroof["frac"] = qroof["achieved"] / peak

    # end to end through the public API: pinned host CSR -> device, build,
    # labels -> pinned host
    e2e = None
    if e2e_steps > 0:
        h_rp = torch.from_numpy(g.off).pin_memory()
        h_col = torch.from_numpy(g.col).pin_memory()
        h_o = torch.from_numpy(order).pin_memory()
        h2d = h_rp.numel() * 8 + h_col.numel() * 4 + h_o.numel() * 4
        # pinned host buffers for the labels, allocated once (like a server's
        # reusable result buffers): off int64[n+1], hub int32[T], dist uint8[T]
        h_off = torch.empty(g.n + 1, dtype=torch.int64, pin_memory=True)
        h_hub = torch.empty(n_labels, dtype=torch.int32, pin_memory=True)
        h_dist = torch.empty(n_labels, dtype=torch.uint8, pin_memory=True)
        d2h = h_off.numel() * 8 + h_hub.numel() * 4 + h_dist.numel()
        e2e_ms, phases = [], []
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        for k in range(e2e_steps + 1):  # the first iteration is a warm-up
            flush.zero_()
            torch.cuda.synchronize(dev)
            t = time.perf_counter()
            ev[0].record(stream)
            d_rp = h_rp.to(dev, non_blocking=True)
            d_col = h_col.to(dev, non_blocking=True)
            d_o = h_o.to(dev, non_blocking=True)
            ev[1].record(stream)
            lab = plb.build(d_rp, d_col, d_o, opts)
            ev[2].record(stream)
            off_d, hub_d, dist_d = lab.device_arrays()
            h_off.copy_(off_d, non_blocking=True)
            h_hub.copy_(hub_d, non_blocking=True)
            h_dist.copy_(dist_d, non_blocking=True)
            ev[3].record(stream)
            torch.cuda.synchronize(dev)
            if k > 0:
                e2e_ms.append(1e3 * (time.perf_counter() - t))
                phases.append([ev[i].elapsed_time(ev[i + 1]) for i in range(3)])
            lab.free()
            del d_rp, d_col, d_o
        e2e_ms_med = max_over_ranks(statistics.median(e2e_ms), world)
        e2e = {"value": whole_job_rate(g.m, e2e_ms_med, world), "unit": "edges/s", "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h, "ms_per_step": e2e_ms_med,
               "phases_ms": {k: statistics.median(x[i] for x in phases) for i, k in enumerate(("h2d", "build", "d2h"))}}
        del h_off, h_hub, h_dist
    del flush, rp, col, o
    plb.release_cached_memory()
    torch.cuda.empty_cache()
    return {"ms": ms, "ms_max": ms_max, "n_labels": n_labels, "rounds": st0["rounds"], "launches": launches,
            "wall": wall, "clocks": clk.summary(), "roofline": roof, "e2e": e2e, "memory": memory,
            "kernel_ms": {"prepare": st["ms_prepare"], "frontier": st["ms_frontier"],
                          "gather_prune": st["ms_gather_prune"][:2], "merge_sort_index": st["ms_merge"],
                          "finalize": st["ms_finalize"]},
            "counters": {k: st[k] for k in ("receivers", "messages_round", "unique_round", "prefiltered_round",
                                            "probed_round", "accepted", "tier_vertices", "launches",
                                            "check_lv_entries", "check_lh_entries")},
            "queries": {"value": q_value, "unit": "queries/s", "batch": 1 << 16,
                        "kernel_p50_ms": qms[len(qms) // 2], "kernel_p99_ms": qms[min(len(qms) - 1, int(0.99 * len(qms)))],
                        "roofline": qroof}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="rmat22")
    ap.add_argument("--batch-hubs", type=int, default=0,
                    help="label in rank batches of this many hubs (Alg. 4); 0 = one batch (Alg. 3)")
    ap.add_argument("--cpu-seconds", type=float, default=15.0,
                    help="budget of the oracle's prefix sample (both CPU legs)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--mode", default="build", choices=["build", "batch", "serve", "directed", "weighted"])
    ap.add_argument("--directed-scale", type=int, default=20)
    ap.add_argument("--batch-graphs", type=int, default=2000)
    ap.add_argument("--serve-resident", default="rmat22")
    ap.add_argument("--serve-seconds", type=float, default=6.0)
    ap.add_argument("--serve-rates", type=float, nargs="+",
                    default=[250.0, 500.0, 1000.0, 1500.0, 2000.0, 2500.0, 3000.0, 4000.0])
    ap.add_argument("--serve-jobs", type=int, default=400)
    ap.add_argument("--serve-job-interval", type=float, default=0.02)
    ap.add_argument("--no-parity-check", action="store_true")
    ap.add_argument("--sub", default="chunglu20,batch,serve",
                    help="sub-objects of the default line (comma list of chunglu20, batch, serve; '' for none)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.mode == "batch":
        return run_batch(args)
    if args.mode == "serve":
        return run_serve(args)
    if args.mode == "directed":
        return run_directed(args)
    if args.mode == "weighted":
        return run_weighted(args)

    import torch

    from paper_1906_12018_gb300 import graphs as G

    world, rank, local = dist_init()
    dev = torch.device("cuda", local if world > 1 else 0)
    g = G.workload(args.workload)
    order = G.degree_order(g)
    warmup = max(args.warmup, 3)
    res = measure_build(args, g, order, dev, args.steps, warmup, args.e2e_steps, world, local)

    subs = {}
    want = [x for x in args.sub.split(",") if x] if world == 1 and rank == 0 else []
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        total = oracle_total_labels(args.workload)
        if total is not None:
            cpu = pll_sample(g, order, total, args.cpu_seconds)
            full = oracle_full_run(args.workload)
            if full and full.get("seconds"):
                cpu["full_run"] = dict(full, value=g.m / float(full["seconds"]), unit="edges/s")
    if "chunglu20" in want and args.workload != "chunglu20":
        g2 = G.workload("chunglu20")
        o2 = G.degree_order(g2)
        a2 = argparse.Namespace(**vars(args))
        a2.workload = "chunglu20"
        r2 = measure_build(a2, g2, o2, dev, 20, 3, args.e2e_steps)
        sub = {"workload": "chunglu20", "n": g2.n, "m": g2.m, "labels": r2["n_labels"], "rounds": r2["rounds"],
               "value": g2.m / (r2["ms"] / 1e3), "unit": "edges/s", "ms_per_step": r2["ms"], "steps": 20,
               "warmup": 3, "roofline": r2["roofline"], "e2e": r2["e2e"], "kernel_ms": r2["kernel_ms"],
               "queries": r2["queries"], "clocks": r2["clocks"], "gpu_launches": r2["launches"]}
        if not args.no_cpu_baseline:
            sub["cpu_baseline"] = pll_full(g2, o2)
        subs["chunglu20"] = sub
    if "batch" in want:
        subs["batch"] = batch_report(args, 2, 1, not args.no_cpu_baseline)
    if "serve" in want and args.workload == args.serve_resident:
        from paper_1906_12018_gb300 import plb

        base = plb.build(torch.from_numpy(g.off).to(dev), torch.from_numpy(g.col).to(dev),
                         torch.from_numpy(order).to(dev))
        subs["serving"] = serve_report(args, base, g, [500.0, 1000.0, 2000.0, 2500.0, 3000.0], 4.0)
        base.free()

    if rank == 0:
        value = whole_job_rate(g.m, res["ms_max"], world)
        line = {
            "metric": "labeling edges/sec",
            "value": value,
            "unit": "edges/s",
            "n_gpus": world,
            "steps": args.steps,
            "warmup": warmup,
            "ms_per_step": res["ms_max"],
            "higher_is_better": True,
            "scaling": "weak",
            "vs_baseline": None,
            "dtype": "int32",
            "data": "synthetic",
            "config": dict(workload_config(args.workload, g, res["n_labels"]), rounds=res["rounds"],
                           parallelism="replicas" if world > 1 else "single", batch_hubs=args.batch_hubs),
            "roofline": res["roofline"],
            "kernel_ms": res["kernel_ms"],
            "counters": res["counters"],
            "e2e": res["e2e"],
            "queries": res["queries"],
            "memory": res["memory"],
            "gpu_launches": res["launches"],
            "clocks": res["clocks"],
            "wall_s_timed": res["wall"],
            "cpu_baseline": cpu,
        }
        line.update(subs)
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
