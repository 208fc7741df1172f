"""Serving policy (no GPU): footprint admission and query coalescing."""
from dataclasses import dataclass

import numpy as np

from paper_1906_12018_gb300.serve import admit_jobs, build_footprint, estimated_labels, plan_query_batch


@dataclass
class J:
    footprint: int


@dataclass
class R:
    num_pairs: int


def test_admission_is_fifo_and_bounded():
    jobs = [J(40), J(30), J(50), J(5)]
    assert admit_jobs(jobs, free_slots=4, budget=100, used=0) == jobs[:2]        # 50 does not fit: stop
    assert admit_jobs(jobs, free_slots=1, budget=1000, used=0) == jobs[:1]       # slot-bound
    assert admit_jobs(jobs, free_slots=4, budget=100, used=70) == []             # head blocks (no overtaking)
    assert admit_jobs([], free_slots=2, budget=10, used=0) == []


def test_query_batches_fill_up_to_the_pair_budget():
    reqs = [R(10), R(20), R(40), R(5)]
    assert plan_query_batch(reqs, 35) == reqs[:2]
    assert plan_query_batch(reqs, 1000) == reqs
    assert plan_query_batch([R(5000), R(1)], 100) == [R(5000)]                  # oversized request goes alone
    assert plan_query_batch([], 100) == []


def test_footprint_grows_with_the_graph():
    a = build_footprint(1000, 8000)
    b = build_footprint(2000, 8000)
    c = build_footprint(2000, 16000)
    assert 0 < a < b < c
    # at least the inputs plus 64 bytes per estimated label
    assert a > 64 * estimated_labels(1000, 8000) + 8 * 1001 + 4 * 8000


# ------------------------------------------------- scheduler, on the host
import contextlib  # noqa: E402
import threading  # noqa: E402
import time  # noqa: E402

import pytest  # noqa: E402

from paper_1906_12018_gb300.serve import LabelServer, estimated_labels  # noqa: E402


class _Stream:
    def synchronize(self):
        pass


class _Cuda:
    def set_device(self, d):
        pass

    def mem_get_info(self, d=None):
        return (1 << 40, 1 << 40)

    def Stream(self, device=None):
        return _Stream()

    @contextlib.contextmanager
    def stream(self, s):
        yield


class _Tensor:
    def __init__(self, a):
        self.a = a

    def to(self, *a, **k):
        return self


class FakeTorch:
    """The pieces of torch the build path of the server touches."""
    cuda = _Cuda()

    def device(self, *a):
        return ("cuda", 0)

    def from_numpy(self, a):
        return _Tensor(a)


class FakeLabels:
    def __init__(self, nbytes):
        self._n = nbytes
        self.freed = False

    def nbytes(self):
        return self._n

    def free(self):
        self.freed = True


class FakePlb:
    """Builds succeed after a delay unless their graph's vertex count is in
    `oom` (a device allocation failure, PLB_ERR_OOM, for the first
    `oom[n]` attempts) or in `broken` (another error)."""
    PLB_ERR_OOM = 2

    class PLBError(RuntimeError):
        def __init__(self, code):
            super().__init__(f"status {code}")
            self.code = code

    def __init__(self, oom=None, broken=(), delay=0.02):
        self.oom = dict(oom or {})
        self.broken = set(broken)
        self.delay = delay
        self.lock = threading.Lock()
        self.running = 0
        self.max_running = 0
        self.attempts = {}

    def build(self, rp, col, o, opts, stream=None):
        n = len(rp.a) - 1
        with self.lock:
            self.attempts[n] = self.attempts.get(n, 0) + 1
            self.running += 1
            self.max_running = max(self.max_running, self.running)
        try:
            time.sleep(self.delay)
            if n in self.broken:
                raise RuntimeError("broken build")
            with self.lock:
                if self.oom.get(n, 0) > 0:
                    self.oom[n] -= 1
                    raise self.PLBError(self.PLB_ERR_OOM)
            return FakeLabels(100 * n)
        finally:
            with self.lock:
                self.running -= 1


def _graph(n):
    off = np.arange(n + 1, dtype=np.int64) * 0
    return off, np.zeros(0, np.int32), np.arange(n, dtype=np.int32)


def _server(plb, budget, slots=2):
    return LabelServer(hbm_budget=budget, build_slots=slots, torch_module=FakeTorch(), plb_module=plb)


def test_label_estimate_matches_the_batched_workload():
    import json
    import os

    with open(os.path.join(os.path.dirname(__file__), "golden", "batch2000_labels.json")) as f:
        gs = json.load(f)["graphs"]
    ratios = [g["labels"] / estimated_labels(g["n"], 2 * g["m"]) for g in gs]
    assert 0.85 < min(ratios) and max(ratios) < 1.25


def test_budget_bounds_running_builds_and_every_job_completes():
    plb = FakePlb()
    fp = build_footprint(1000, 0)
    srv = _server(plb, budget=int(2.5 * fp), slots=4)   # two footprints fit, not three
    try:
        futs = [srv.submit_build(f"g{i}", *_graph(1000)) for i in range(6)]
        srv.wait_idle(timeout=30)
        assert all(f.result().nbytes() == 100 * 1000 for f in futs)
        assert plb.max_running == 2                        # admission by footprint, not by slots
        assert srv.peak_used <= srv.budget
    finally:
        srv.close()


def test_job_that_can_never_fit_is_rejected_and_does_not_block_the_queue():
    plb = FakePlb()
    srv = _server(plb, budget=build_footprint(1000, 0) + 10)
    try:
        big = srv.submit_build("big", *_graph(100_000))
        q = srv.submit_query("big", np.zeros((3, 2), np.int32))
        small = srv.submit_build("small", *_graph(1000))
        srv.wait_idle(timeout=30)
        with pytest.raises(MemoryError):
            big.result()
        with pytest.raises(MemoryError):
            q.future.result()
        assert small.result().nbytes() == 100 * 1000
    finally:
        srv.close()


def test_out_of_memory_build_is_requeued_then_runs():
    plb = FakePlb(oom={1000: 1})
    srv = _server(plb, budget=1 << 40)
    try:
        f = srv.submit_build("g", *_graph(1000))
        srv.wait_idle(timeout=30)
        assert f.result().nbytes() == 100 * 1000
        assert plb.attempts[1000] == 2
    finally:
        srv.close()


def test_failed_build_fails_its_queued_queries():
    plb = FakePlb(broken={1000}, oom={2000: 10})
    srv = _server(plb, budget=1 << 40)
    try:
        f1 = srv.submit_build("a", *_graph(1000))
        q1 = srv.submit_query("a", np.zeros((2, 2), np.int32))
        f2 = srv.submit_build("b", *_graph(2000))          # out of memory on every attempt
        q2 = srv.submit_query("b", np.zeros((2, 2), np.int32))
        srv.wait_idle(timeout=30)
        for f in (f1, q1.future):
            with pytest.raises(RuntimeError):
                f.result()
        for f in (f2, q2.future):
            with pytest.raises(FakePlb.PLBError):
                f.result()
        assert plb.attempts[2000] == 1 + srv.max_oom_retries
        assert not srv.pending_queries
    finally:
        srv.close()


def test_duplicate_names_and_unknown_sets_are_refused():
    plb = FakePlb()
    srv = _server(plb, budget=1 << 40)
    try:
        srv.add_resident("base", FakeLabels(10))
        with pytest.raises(ValueError):
            srv.add_resident("base", FakeLabels(10))
        with pytest.raises(ValueError):
            srv.submit_build("base", *_graph(10)).result()
        f = srv.submit_build("x", *_graph(10))
        with pytest.raises(ValueError):
            srv.submit_build("x", *_graph(10)).result()     # queued or running
        with pytest.raises(KeyError):
            srv.submit_query("nope", np.zeros((1, 2), np.int32)).future.result()
        srv.wait_idle(timeout=30)
        assert f.result().nbytes() == 1000
        assert srv.used == 10 + 1000
    finally:
        srv.close()
