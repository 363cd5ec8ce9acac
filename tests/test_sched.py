"""Admission policy of the worker pool (host logic, no GPU): the discrete-event
simulator tlr_sched_simulate runs the same admission class the pool uses.

Checked: the HBM budget is never exceeded; the requests of one dataset run one
at a time in arrival order; with room for everything the schedule is the
work-conserving FIFO schedule (against a plain re-statement below); idle
factors are evicted least recently used first; a request waiting for memory is
not overtaken by later allocating requests; datasets that cannot fit are
refused."""
import heapq

import numpy as np
import pytest

import paper_2402_09356_gb300 as tlr
from paper_2402_09356_gb300 import build as tlr_build


@pytest.fixture(scope="module", autouse=True)
def lib():
    tlr_build.build()
    return tlr.load_library()


def fifo_schedule(workers, req_data, arrival, cost):
    """Work-conserving FIFO with one running request per dataset and no memory
    limit: at each event, start queued requests in arrival order while a
    worker is free, skipping requests whose dataset is running."""
    n = len(req_data)
    start = np.full(n, np.nan)
    finish = np.full(n, np.nan)
    queue, running, busy = [], [], set()
    nxt, now, done = 0, 0.0, 0
    while done < n:
        for q in list(queue):
            if len(running) >= workers:
                break
            if req_data[q] in busy:
                continue
            queue.remove(q)
            busy.add(req_data[q])
            start[q], finish[q] = now, now + cost[q]
            heapq.heappush(running, (finish[q], q))
        t_arr = arrival[nxt] if nxt < n else np.inf
        t_fin = running[0][0] if running else np.inf
        if t_fin <= t_arr:
            now, q = heapq.heappop(running)
            busy.discard(req_data[q])
            done += 1
        else:
            now = t_arr
            queue.append(nxt)
            nxt += 1
    return start, finish


def random_trace(rng, ndata, nreq):
    req = rng.integers(0, ndata, nreq).astype(np.int32)
    arr = np.cumsum(rng.exponential(0.3, nreq))
    cost = rng.uniform(0.1, 2.0, nreq)
    return req, arr, cost


@pytest.mark.parametrize("seed", range(5))
def test_unlimited_budget_is_fifo(seed):
    rng = np.random.default_rng(seed)
    ndata, nreq, workers = 7, 120, 3
    req, arr, cost = random_trace(rng, ndata, nreq)
    base = np.full(ndata, 10)
    fb = rng.integers(100, 1000, ndata)
    wb = rng.integers(10, 100, ndata)
    start, finish, peak, ev = tlr.tlr_sched_simulate(10**12, workers, base, fb, wb, req, arr, cost)
    s2, f2 = fifo_schedule(workers, req, arr, cost)
    np.testing.assert_array_equal(start, s2)
    np.testing.assert_array_equal(finish, f2)
    assert ev == 0
    assert peak <= base.sum() + fb.sum() + wb.sum()


@pytest.mark.parametrize("seed", range(8))
def test_budget_and_per_dataset_order(seed):
    rng = np.random.default_rng(100 + seed)
    ndata, nreq, workers = 9, 200, 4
    req, arr, cost = random_trace(rng, ndata, nreq)
    base = rng.integers(1, 20, ndata)
    fb = rng.integers(50, 400, ndata)
    wb = rng.integers(5, 60, ndata)
    budget = int(base.sum() + (fb + wb).max() + rng.integers(0, 600))
    start, finish, peak, ev = tlr.tlr_sched_simulate(budget, workers, base, fb, wb, req, arr, cost)
    assert peak <= budget
    assert np.all(start >= arr - 1e-12)
    # at most `workers` requests at once
    events = sorted([(s, 1) for s in start] + [(f, -1) for f in finish], key=lambda e: (e[0], e[1]))
    live = 0
    for _, d in events:
        live += d
        assert live <= workers
    # one dataset: arrival order, never overlapping
    for d in range(ndata):
        idx = np.nonzero(req == d)[0]
        assert np.all(np.diff(start[idx]) >= 0)
        assert np.all(start[idx][1:] >= finish[idx][:-1] - 1e-12)


def test_lru_eviction():
    # room for two factors; A, B, A, C, A on one worker: LRU evicts B for C (1
    # eviction); evicting the oldest allocation (A) would cost a second one
    base, fb, wb = [0, 0, 0], [100, 100, 100], [0, 0, 0]
    req = [0, 1, 0, 2, 0]
    arr = [0, 0, 0, 0, 0]
    cost = [1, 1, 1, 1, 1]
    start, finish, peak, ev = tlr.tlr_sched_simulate(200, 1, base, fb, wb, req, arr, cost)
    assert ev == 1
    assert peak == 200
    np.testing.assert_array_equal(start, [0, 1, 2, 3, 4])


def test_waiting_request_not_overtaken_by_later_allocations():
    # budget 100: small datasets (30) and a big one (100).  small0 runs; the big
    # request cannot fit until small0's factor is evicted after it ends; the
    # later small1 request must not jump ahead of it.
    base, fb, wb = [0, 0, 0], [30, 100, 30], [0, 0, 0]
    req = [0, 1, 2]
    arr = [0.0, 0.1, 0.2]
    cost = [5.0, 1.0, 1.0]
    start, finish, peak, ev = tlr.tlr_sched_simulate(100, 2, base, fb, wb, req, arr, cost)
    assert start[1] == 5.0  # after small0 finished and was evicted
    assert start[2] == finish[1] == 6.0
    assert peak <= 100
    assert ev == 2


def test_resident_factor_runs_beside_a_waiting_allocation():
    # dataset 0 is resident and idle; the big request waits for memory; a new
    # request of dataset 0 needs no allocation and may run meanwhile
    base, fb, wb = [0, 0, 0], [40, 100, 40], [0, 0, 0]
    req = [0, 2, 1, 0]
    arr = [0.0, 0.0, 0.5, 0.6]
    cost = [1.0, 10.0, 1.0, 1.0]
    start, finish, peak, ev = tlr.tlr_sched_simulate(100, 3, base, fb, wb, req, arr, cost)
    np.testing.assert_array_equal(start, [0.0, 0.0, 10.0, 1.0])
    assert peak <= 100
    assert ev == 2


def test_dataset_too_large_is_refused():
    with pytest.raises(tlr.TlrError) as e:
        tlr.tlr_sched_simulate(100, 2, [10, 10], [50, 85], [5, 5], [0], [0.0], [1.0])
    assert e.value.code == tlr.TLR_ERR_OOM


def test_bad_arguments():
    with pytest.raises(tlr.TlrError):
        tlr.tlr_sched_simulate(100, 0, [1], [1], [1], [0], [0.0], [1.0])
    with pytest.raises(tlr.TlrError):
        tlr.tlr_sched_simulate(100, 1, [1], [1], [1], [3], [0.0], [1.0])
    with pytest.raises(tlr.TlrError):
        tlr.tlr_sched_simulate(100, 1, [1], [1], [1], [0, 0], [1.0, 0.0], [1.0, 1.0])


def test_pool_creation_fails_cleanly_without_gpu():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(tlr.TlrError):
        tlr.Pool(0, workers=2, nb=256)
    with pytest.raises(tlr.TlrError):
        tlr.Pool(0, workers=0, nb=256)
