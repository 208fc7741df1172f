"""Serving policy (no GPU): footprint admission and query coalescing."""
from dataclasses import dataclass

import numpy as np

from paper_1906_12018_gb300.serve import admit_jobs, build_footprint, plan_query_batch


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
    # at least the final labels of ~96 entries per vertex plus the inputs
    assert a > 9 * 96 * 1000 + 8 * 1001 + 4 * 8000
