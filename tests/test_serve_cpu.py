"""Serving scheduler logic on the CPU: admission by slots and device-memory budget."""
import threading
import time

import numpy as np
import pytest

from paper_1606_03135_gb300 import serve as S


def test_budget_never_exceeds_slots_or_bytes():
    b = S.Budget(slots=3, budget_bytes=100)
    live = {"jobs": 0, "bytes": 0, "max_jobs": 0, "max_bytes": 0}
    lock = threading.Lock()

    def job(need, hold):
        b.admit(need)
        with lock:
            live["jobs"] += 1
            live["bytes"] += need
            live["max_jobs"] = max(live["max_jobs"], live["jobs"])
            live["max_bytes"] = max(live["max_bytes"], live["bytes"])
        time.sleep(hold)
        with lock:
            live["jobs"] -= 1
            live["bytes"] -= need
        b.release(need)

    sizes = [40, 30, 50, 20, 60, 10, 45, 35, 25, 55]
    ts = [threading.Thread(target=job, args=(s, 0.01 * (1 + i % 3))) for i, s in enumerate(sizes)]
    for t in ts:
        t.start()
    for t in ts:
        t.join(30)
    assert live["max_jobs"] <= 3 and live["max_bytes"] <= 100
    assert b.in_use == 0 and b.free_slots == 3


def test_budget_resize_shrinks_and_grows_only_into_free_room():
    b = S.Budget(slots=2, budget_bytes=100)
    b.admit(60)
    b.admit(30)
    b.resize(30, 20)  # the exact size is smaller: room is handed back at once
    assert b.in_use == 80
    b.resize(20, 40)  # grows into free room without waiting
    assert b.in_use == 100 and b.peak == 100


def test_budget_resize_never_waits_while_holding_a_slot():
    # two running jobs that both need to grow beyond the budget: each fails at once (the job
    # is reported as failed) instead of waiting for the other
    b = S.Budget(slots=2, budget_bytes=100)
    b.admit(50)
    b.admit(40)
    t0 = time.perf_counter()
    for old, new in ((50, 70), (40, 60)):
        with pytest.raises(MemoryError):
            b.resize(old, new)
    assert time.perf_counter() - t0 < 1.0
    assert b.in_use == 90  # the failed resizes left the reservations as they were
    b.release(50)
    b.release(40)
    assert b.in_use == 0 and b.free_slots == 2


def test_oversized_job_is_refused():
    b = S.Budget(slots=1, budget_bytes=10)
    with pytest.raises(MemoryError):
        b.admit(11)
    assert b.free_slots == 1 and b.in_use == 0


def test_serving_mix_follows_its_recipe():
    jobs = S.serving_jobs(count=24, n_min=1000, n_max=3000)
    assert [j.rid for j in jobs] == list(range(24))
    for j in jobs:
        N, d = j.nodes.shape
        assert d in (2, 3) and 1000 <= N <= 3000
        assert 2 <= j.ell <= 5 and 0.2 <= j.delta <= 1.0
        from math import comb
        assert j.n == 2 * comb(j.ell + d, d) + 1
        assert j.m == (5 if j.ell == 2 else 7)
    again = S.serving_jobs(count=24, n_min=1000, n_max=3000)
    assert all(np.array_equal(a.nodes, b.nodes) for a, b in zip(jobs, again))
    S.poisson_arrivals(jobs, rate=10.0)
    t = np.array([j.arrival for j in jobs])
    assert np.all(np.diff(t) > 0) and 0.5 < t[-1] < 10


def test_estimate_covers_growth():
    a = S.estimate_bytes(10000, 2, 31, 0.5)
    assert a > S.estimate_bytes(10000, 2, 31, 1.0) > 0
    assert S.estimate_bytes(20000, 2, 31, 0.5) > a
