"""Continuous-batching serving loop over resident label sets (one GPU).

* Label sets stay resident on the device, addressed by name.
* Labeling jobs (graph + vertex order) are admitted when a build slot is free
  and their estimated device footprint fits the HBM budget; each admitted job
  runs ``plb_build`` on its own CUDA stream in a worker thread, so builds
  overlap with each other and with query work on the device.  The estimate is
  replaced by the measured size of the label set when the build finishes.
* Distance-query requests (a set name and int32 [q, 2] pairs) queue up; the
  scheduler coalesces all pending requests (up to a pair budget) into ONE
  ``plb_query_multi`` launch on the query stream, with up to
  ``max_inflight`` launches in flight, so requests that arrive while a launch
  runs join the next one.
* Latency of a request = arrival (submit) -> its distances on the host.

The policy pieces (``admit_jobs``, ``plan_query_batch``, ``build_footprint``)
are pure functions; the CUDA work all goes through the C ABI binding.
"""
from __future__ import annotations

import collections
import threading
import time
from concurrent.futures import Future, ThreadPoolExecutor
from dataclasses import dataclass, field

import numpy as np


# ------------------------------------------------------------------ policy
def build_footprint(n: int, nnz: int, label_bytes_per_vertex: int = 9 * 96) -> int:
    """Conservative device bytes of a build of a graph with n vertices and nnz
    arcs: inputs (8(n+1) + 4 nnz + 4n), rank-space copy and frontier buffers
    (about 3x the arcs), label buffers during the build (two copies and the
    probe index) and the final labels, at ``label_bytes_per_vertex`` per
    vertex, plus the 256-byte top-hub row per vertex."""
    inputs = 8 * (n + 1) + 4 * nnz + 4 * n
    work = 12 * nnz + 64 * n
    labels = 4 * label_bytes_per_vertex * n
    return int(inputs + work + labels + 256 * n)


def admit_jobs(pending: list, free_slots: int, budget: int, used: int) -> list:
    """FIFO admission: take jobs from the head while a slot is free and the
    job's footprint fits in budget - used; stop at the first that does not fit
    (no overtaking, so a large job is not starved)."""
    admitted = []
    for job in pending:
        if free_slots <= 0 or used + job.footprint > budget:
            break
        admitted.append(job)
        used += job.footprint
        free_slots -= 1
    return admitted


def plan_query_batch(pending: list, max_pairs: int) -> list:
    """Requests (FIFO) coalesced into one launch: as many as fit in max_pairs,
    and always at least one (a request larger than max_pairs goes alone)."""
    out, total = [], 0
    for r in pending:
        q = r.num_pairs
        if out and total + q > max_pairs:
            break
        out.append(r)
        total += q
    return out


# ------------------------------------------------------------------ requests
@dataclass
class QueryRequest:
    set_name: str
    pairs: np.ndarray                 # int32 [q, 2]
    t_submit: float = 0.0
    t_done: float = 0.0
    result: np.ndarray | None = None
    future: Future = field(default_factory=Future)

    @property
    def num_pairs(self) -> int:
        return int(self.pairs.shape[0])

    @property
    def latency(self) -> float:
        return self.t_done - self.t_submit


@dataclass
class BuildJob:
    name: str
    off: np.ndarray
    col: np.ndarray
    order: np.ndarray
    footprint: int
    t_submit: float = 0.0
    t_done: float = 0.0
    future: Future = field(default_factory=Future)


# ------------------------------------------------------------------ server
class LabelServer:
    def __init__(self, device: int = 0, hbm_budget: int | None = None, build_slots: int = 2,
                 max_inflight: int = 2, max_pairs_per_launch: int = 1 << 21, options=None):
        import torch

        from . import plb

        self.torch = torch
        self.plb = plb
        self.device = torch.device("cuda", device)
        torch.cuda.set_device(self.device)
        free, total = torch.cuda.mem_get_info(self.device)
        self.budget = int(hbm_budget if hbm_budget is not None else 0.8 * free)
        self.used = 0
        self.sets: dict[str, object] = {}
        self.set_bytes: dict[str, int] = {}
        self.busy_sets: collections.Counter = collections.Counter()
        self.build_slots = build_slots
        self.running_builds = 0
        self.max_inflight = max_inflight
        self.max_pairs = max_pairs_per_launch
        self.options = options
        self.pending_builds: collections.deque = collections.deque()
        self.pending_queries: collections.deque = collections.deque()
        self.inflight: collections.deque = collections.deque()
        self.lock = threading.Lock()
        self.wake = threading.Condition(self.lock)
        self.pool = ThreadPoolExecutor(max_workers=build_slots)
        self.qstream = torch.cuda.Stream(self.device)
        self.stop_flag = False
        self.completed_queries: list[QueryRequest] = []
        self.completed_builds: list[BuildJob] = []
        self.thread = threading.Thread(target=self._loop, name="plb-scheduler", daemon=True)
        self.thread.start()

    # -------------------------------------------------------------- public
    def add_resident(self, name: str, labels) -> None:
        with self.lock:
            self.sets[name] = labels
            self.set_bytes[name] = labels.nbytes()
            self.used += self.set_bytes[name]

    def submit_build(self, name: str, off: np.ndarray, col: np.ndarray, order: np.ndarray) -> Future:
        job = BuildJob(name, np.ascontiguousarray(off, np.int64), np.ascontiguousarray(col, np.int32),
                       np.ascontiguousarray(order, np.int32),
                       build_footprint(len(off) - 1, len(col)), time.perf_counter())
        with self.wake:
            self.pending_builds.append(job)
            self.wake.notify()
        return job.future

    def submit_query(self, set_name: str, pairs: np.ndarray) -> QueryRequest:
        req = QueryRequest(set_name, np.ascontiguousarray(pairs, np.int32).reshape(-1, 2), time.perf_counter())
        with self.wake:
            self.pending_queries.append(req)
            self.wake.notify()
        return req

    def drop(self, name: str) -> None:
        """Free a resident set once no in-flight query uses it."""
        while True:
            with self.lock:
                if self.busy_sets[name] == 0:
                    lab = self.sets.pop(name)
                    self.used -= self.set_bytes.pop(name)
                    break
            time.sleep(1e-4)
        lab.free()

    def wait_idle(self, timeout: float = 600.0) -> None:
        t0 = time.perf_counter()
        while time.perf_counter() - t0 < timeout:
            with self.lock:
                idle = (not self.pending_builds and not self.pending_queries and not self.inflight
                        and self.running_builds == 0)
            if idle:
                return
            time.sleep(1e-3)
        raise TimeoutError("server did not drain")

    def close(self) -> None:
        with self.wake:
            self.stop_flag = True
            self.wake.notify()
        self.thread.join()
        self.pool.shutdown(wait=True)

    # -------------------------------------------------------------- builds
    def _run_build(self, job: BuildJob) -> None:
        torch, plb = self.torch, self.plb
        try:
            torch.cuda.set_device(self.device)
            stream = torch.cuda.Stream(self.device)
            with torch.cuda.stream(stream):
                rp = torch.from_numpy(job.off).to(self.device, non_blocking=True)
                col = torch.from_numpy(job.col).to(self.device, non_blocking=True)
                o = torch.from_numpy(job.order).to(self.device, non_blocking=True)
                lab = plb.build(rp, col, o, self.options, stream=stream)
                stream.synchronize()
            job.t_done = time.perf_counter()
            with self.wake:
                self.sets[job.name] = lab
                self.set_bytes[job.name] = lab.nbytes()
                self.used += lab.nbytes() - job.footprint
                self.running_builds -= 1
                self.completed_builds.append(job)
                self.wake.notify()
            job.future.set_result(lab)
        except Exception as e:  # reported to the submitter
            with self.wake:
                self.used -= job.footprint
                self.running_builds -= 1
                self.wake.notify()
            job.future.set_exception(e)

    # -------------------------------------------------------------- queries
    def _launch_queries(self, reqs: list) -> None:
        torch, plb = self.torch, self.plb
        names = sorted({r.set_name for r in reqs})
        sets = [self.sets[nm] for nm in names]
        index = {nm: i for i, nm in enumerate(names)}
        q = sum(r.num_pairs for r in reqs)
        pairs_h = torch.empty((q, 2), dtype=torch.int32, pin_memory=True)
        sidx_h = torch.empty(q, dtype=torch.int32, pin_memory=True)
        pos = 0
        bounds = []
        for r in reqs:
            k = r.num_pairs
            pairs_h[pos:pos + k] = torch.from_numpy(r.pairs)
            sidx_h[pos:pos + k] = index[r.set_name]
            bounds.append((pos, pos + k))
            pos += k
        out_h = torch.empty(q, dtype=torch.int32, pin_memory=True)
        with torch.cuda.stream(self.qstream):
            pairs_d = pairs_h.to(self.device, non_blocking=True)
            sidx_d = sidx_h.to(self.device, non_blocking=True)
            out_d = torch.empty(q, dtype=torch.int32, device=self.device)
            plb.query_multi(sets, sidx_d, pairs_d, out_d, stream=self.qstream)
            out_h.copy_(out_d, non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(self.qstream)
        for nm in names:
            self.busy_sets[nm] += 1
        # keep the device buffers alive until the event completes
        self.inflight.append((ev, reqs, bounds, out_h, names, (pairs_d, sidx_d, out_d, pairs_h, sidx_h)))

    def _retire_queries(self) -> bool:
        done_any = False
        while self.inflight and self.inflight[0][0].query():
            ev, reqs, bounds, out_h, names, _keep = self.inflight.popleft()
            now = time.perf_counter()
            res = out_h.numpy()
            for r, (a, b) in zip(reqs, bounds):
                r.result = res[a:b].copy()
                r.t_done = now
                r.future.set_result(r.result)
            self.completed_queries.extend(reqs)
            for nm in names:
                self.busy_sets[nm] -= 1
            done_any = True
        return done_any

    # -------------------------------------------------------------- scheduler
    def _loop(self) -> None:
        self.torch.cuda.set_device(self.device)
        while True:
            with self.wake:
                if self.stop_flag:
                    return
                # admit labeling jobs
                admitted = admit_jobs(list(self.pending_builds), self.build_slots - self.running_builds,
                                      self.budget, self.used)
                for job in admitted:
                    self.pending_builds.popleft()
                    self.used += job.footprint
                    self.running_builds += 1
                    self.pool.submit(self._run_build, job)
                # coalesce ready query requests (their set must be resident)
                batch = []
                if len(self.inflight) < self.max_inflight and self.pending_queries:
                    ready = [r for r in self.pending_queries if r.set_name in self.sets]
                    batch = plan_query_batch(ready, self.max_pairs)
                    for r in batch:
                        self.pending_queries.remove(r)
                    if batch:
                        self._launch_queries(batch)
                progressed = bool(admitted) or bool(batch)
            progressed = self._retire_queries() or progressed
            if not progressed:
                with self.wake:
                    if not self.stop_flag:
                        self.wake.wait(timeout=2e-4)


def latency_summary(reqs: list) -> dict:
    lat = np.array([r.latency for r in reqs]) * 1e3
    pairs = int(sum(r.num_pairs for r in reqs))
    if not len(lat):
        return {"requests": 0}
    t0 = min(r.t_submit for r in reqs)
    t1 = max(r.t_done for r in reqs)
    return {"requests": len(reqs), "pairs": pairs, "queries_per_s": pairs / max(t1 - t0, 1e-9),
            "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "mean_ms": float(lat.mean())}
