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
# Label count of a graph, fitted (least squares on log(labels / n)) to the
# oracle's label totals of the 2,000 graphs of the batched workload: within
# -11% .. +19% of every one of them; the R-MAT scale-22 graph has 1.43x the
# model's count, so estimates carry a safety factor.
LABELS_LOG_COEF = (-0.6997, 0.3050, 0.7563)  # log(labels/n) = a + b log n + c log(nnz/2n)
LABEL_SAFETY = 1.5
# Device bytes per final label at a build's peak (label buffers of both
# parities, the probe tables, the frontier buffers): the R-MAT scale-22 build
# peaks at 74.8 GB, 38 bytes per label beyond its per-vertex and per-arc
# buffers (measured with plb_memory_stats).
BUILD_BYTES_PER_LABEL = 64
# Resident blocks of the block tier (152 SMs x 3), each holding one n-word
# row of the labels it accepts for a vertex.
GATHER_BLOCKS = 456
# Per-vertex device bytes of a build's round state: rank inverse and CSR
# offsets, label and frontier offsets (two parities), lists, bounds and
# cursors, the 224-byte top-hub masks, probe-index offsets and descriptors,
# check records and the row-sort scratch (8 rows of the next power of two).
BUILD_BYTES_PER_VERTEX = 440


def estimated_labels(n: int, nnz: int) -> float:
    """Label count estimate of a graph with n vertices and nnz arcs (nnz/2
    undirected edges), before the safety factor."""
    import math

    if n <= 0:
        return 0.0
    a, b, c = LABELS_LOG_COEF
    deg = max(nnz / 2.0 / n, 0.5)
    return n * math.exp(a + b * math.log(n) + c * math.log(deg))


def build_footprint(n: int, nnz: int) -> int:
    """Device bytes a build of this graph is expected to hold at its peak:
    inputs (8(n+1) + 4 nnz + 4n), the rank-space CSR and first frontier
    buffers (12 bytes per arc), the round state (BUILD_BYTES_PER_VERTEX and
    the block tier's accepted rows, 4 GATHER_BLOCKS bytes per vertex), 1 MiB
    of fixed scratch, and BUILD_BYTES_PER_LABEL per estimated label (with the
    safety factor)."""
    inputs = 8 * (n + 1) + 4 * nnz + 4 * n
    work = 12 * nnz + (BUILD_BYTES_PER_VERTEX + 4 * GATHER_BLOCKS) * n + (1 << 20)
    labels = BUILD_BYTES_PER_LABEL * LABEL_SAFETY * estimated_labels(n, nnz)
    return int(inputs + work + labels)


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
    retries: int = 0                  # re-admissions after the device ran out of memory


# ------------------------------------------------------------------ server
class LabelServer:
    def __init__(self, device: int = 0, hbm_budget: int | None = None, build_slots: int = 2,
                 max_inflight: int = 2, max_pairs_per_launch: int = 1 << 21, options=None,
                 torch_module=None, plb_module=None):
        """torch_module / plb_module replace torch and the library binding
        (host-side tests of the scheduling drive it with fakes)."""
        if torch_module is None:
            import torch as torch_module
        if plb_module is None:
            from . import plb as plb_module
        torch = torch_module
        self.torch = torch
        self.plb = plb_module
        self.device = torch.device("cuda", device)
        torch.cuda.set_device(self.device)
        free, total = torch.cuda.mem_get_info(self.device)
        self.budget = int(hbm_budget if hbm_budget is not None else 0.8 * free)
        self.used = 0
        self.peak_used = 0                # largest admitted total (resident sets + running footprints)
        self.sets: dict[str, object] = {}
        self.set_bytes: dict[str, int] = {}
        self.busy_sets: collections.Counter = collections.Counter()
        self.build_slots = build_slots
        self.running_builds = 0
        self.running_names: set[str] = set()
        self.max_oom_retries = 2
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
            if self._known(name):
                raise ValueError(f"label set {name!r} exists or is being built")
            self.sets[name] = labels
            self.set_bytes[name] = labels.nbytes()
            self.used += self.set_bytes[name]

    def _known(self, name: str) -> bool:
        """A set of this name is resident, queued or being built (lock held)."""
        return (name in self.sets or name in self.running_names
                or any(j.name == name for j in self.pending_builds))

    def submit_build(self, name: str, off: np.ndarray, col: np.ndarray, order: np.ndarray) -> Future:
        """Queue a labeling job.  A name already resident, queued or being
        built is refused (the future fails with ValueError): replacing a
        resident set in place would leak it."""
        job = BuildJob(name, np.ascontiguousarray(off, np.int64), np.ascontiguousarray(col, np.int32),
                       np.ascontiguousarray(order, np.int32),
                       build_footprint(len(off) - 1, len(col)), time.perf_counter())
        with self.wake:
            if self._known(name):
                job.future.set_exception(ValueError(f"label set {name!r} exists or is being built"))
                return job.future
            self.pending_builds.append(job)
            self.wake.notify()
        return job.future

    def submit_query(self, set_name: str, pairs: np.ndarray) -> QueryRequest:
        """Queue a distance-query request on a resident set or on one whose
        build is queued or running (it waits for the build).  A request on an
        unknown name fails at once (KeyError on its future)."""
        req = QueryRequest(set_name, np.ascontiguousarray(pairs, np.int32).reshape(-1, 2), time.perf_counter())
        with self.wake:
            if not self._known(set_name):
                req.t_done = time.perf_counter()
                req.future.set_exception(KeyError(set_name))
                return req
            self.pending_queries.append(req)
            self.wake.notify()
        return req

    def _fail_queries(self, name: str, exc: BaseException) -> None:
        """Fail every queued request on `name` (lock held)."""
        now = time.perf_counter()
        keep = collections.deque()
        for r in self.pending_queries:
            if r.set_name == name:
                r.t_done = now
                r.future.set_exception(exc)
            else:
                keep.append(r)
        self.pending_queries = keep

    def _reject(self, job: BuildJob, exc: BaseException) -> None:
        """The job will never run: fail it and the requests waiting for it (lock held)."""
        job.t_done = time.perf_counter()
        job.future.set_exception(exc)
        self._fail_queries(job.name, exc)

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
            self._build_hook(job)
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
                self.running_names.discard(job.name)
                self.completed_builds.append(job)
                self.wake.notify()
            job.future.set_result(lab)
        except Exception as e:  # reported to the submitter
            oom = isinstance(e, plb.PLBError) and e.code == plb.PLB_ERR_OOM
            with self.wake:
                self.used -= job.footprint
                self.running_builds -= 1
                self.running_names.discard(job.name)
                if oom and job.retries < self.max_oom_retries:
                    # the estimate was too small, or other work held the
                    # memory: wait for twice the footprint and run it again
                    job.retries += 1
                    job.footprint = 2 * job.footprint
                    self.pending_builds.appendleft(job)
                else:
                    self._reject(job, e)
                self.wake.notify()

    def _build_hook(self, job: BuildJob) -> None:
        """Called in the worker before each build attempt (tests inject
        failures here)."""

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
                # a job at the head that cannot fit even once every running
                # build has finished (only resident sets hold memory then)
                # is rejected, so that it does not block the queue for good
                resident = sum(self.set_bytes.values())
                while self.pending_builds and self.pending_builds[0].footprint > self.budget - resident:
                    job = self.pending_builds.popleft()
                    self._reject(job, MemoryError(
                        f"build {job.name!r} needs about {job.footprint} bytes; the budget leaves "
                        f"{self.budget - resident} beside the resident sets"))
                # admit labeling jobs
                admitted = admit_jobs(list(self.pending_builds), self.build_slots - self.running_builds,
                                      self.budget, self.used)
                for job in admitted:
                    self.pending_builds.popleft()
                    self.used += job.footprint
                    self.running_builds += 1
                    self.running_names.add(job.name)
                    self.peak_used = max(self.peak_used, self.used)
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
                        # launches in flight are polled (their CUDA events);
                        # otherwise sleep until a submit or a build wakes us
                        self.wake.wait(timeout=2e-4 if self.inflight else 0.05)


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
