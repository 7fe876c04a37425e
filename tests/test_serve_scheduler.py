"""Host-side admission logic of the server (no GPU): FIFO admission by free
slots and a device-memory budget, concurrency bounded by both, oversize
requests rejected, every request completed exactly once."""
import threading
import time

import pytest

from paper_2603_14641_gb300.serve import Request, Result, Scheduler


def _fake(delay_of):
    lock = threading.Lock()
    log = []

    def execute(req, slot, admit, fp):
        with lock:
            log.append(("start", req.rid, slot, admit))
        time.sleep(delay_of(req))
        return Result(req.rid, 0, req.shots, req.arrival_s, admit, 0.0, fp)

    return execute, log


def _reqs(sizes, gap=0.0):
    return [Request(i, i * gap, None, shots=s, seed=i) for i, s in enumerate(sizes)]


def test_budget_and_slots_bound_concurrency():
    sizes = [30, 50, 20, 70, 10, 40, 60, 25]
    ex, log = _fake(lambda r: 0.02)
    sch = Scheduler(slots=3, budget_bytes=100, footprint=lambda r: r.shots, execute=ex)
    res = sch.run(_reqs(sizes), realtime=False)
    assert sorted(r.rid for r in res) == list(range(len(sizes)))
    assert sch.peak_in_use <= 100
    assert sch.peak_active <= 3
    assert sch.peak_active >= 2  # requests overlapped
    # FIFO: admission order is arrival order
    starts = [rid for kind, rid, _, _ in sorted(log, key=lambda t: t[3])]
    assert starts == sorted(starts)


def test_head_of_line_waits_for_memory():
    # the second request does not fit next to the first; it must wait, not be skipped
    ex, log = _fake(lambda r: 0.05 if r.rid == 0 else 0.01)
    sch = Scheduler(slots=4, budget_bytes=100, footprint=lambda r: r.shots, execute=ex)
    res = sch.run(_reqs([80, 60, 10]), realtime=False)
    by = {r.rid: r for r in res}
    assert by[1].admit_s >= by[0].done_s - 1e-3
    assert by[2].admit_s >= by[1].admit_s


def test_oversize_request_is_rejected():
    ex, _ = _fake(lambda r: 0.0)
    sch = Scheduler(slots=2, budget_bytes=50, footprint=lambda r: r.shots, execute=ex)
    with pytest.raises(MemoryError):
        sch.run(_reqs([10, 500, 10]), realtime=False)


def test_realtime_arrivals_are_respected():
    ex, _ = _fake(lambda r: 0.0)
    sch = Scheduler(slots=2, budget_bytes=1000, footprint=lambda r: r.shots, execute=ex)
    res = sch.run(_reqs([1, 1, 1], gap=0.05), realtime=True)
    for r in res:
        assert r.admit_s >= r.arrival_s - 1e-3


def test_failing_request_releases_its_budget_and_is_reported():
    """An exception in one request reaches the caller of run(); its memory and
    slot are released, so every other request still completes."""
    done = []

    def execute(req, slot, admit, fp):
        if req.rid == 1:
            raise RuntimeError("request 1 failed")
        time.sleep(0.01)
        done.append(req.rid)
        return Result(req.rid, 0, req.shots, req.arrival_s, admit, 0.0, fp)

    sch = Scheduler(slots=2, budget_bytes=100, footprint=lambda r: r.shots, execute=execute)
    with pytest.raises(RuntimeError, match="request 1 failed"):
        sch.run(_reqs([60, 60, 60, 60]), realtime=False)
    assert sorted(done) == [0, 2, 3]
    assert sch.in_use == 0 and sch.active == 0


def test_footprint_and_summary():
    from paper_2603_14641_gb300 import qs
    from paper_2603_14641_gb300.serve import footprint_bytes, summarize
    base = footprint_bytes(1000, 5000, 1000, 1000)
    assert base > qs.qs_sim_required_bytes(1000)
    # frames (2 n words per 64 shots, rounded to 4 words) and records grow with the shots
    more = footprint_bytes(1000, 5000, 1000, 1000 + 256)
    assert more - base == 2 * 1000 * 4 * 8 + 3 * 1000 * 4 * 8
    assert footprint_bytes(2000, 5000, 1000, 1000) > base
    res = [Result(i, 10, 100, 0.0, 0.0, float(i + 1), 0) for i in range(100)]
    s = summarize(res, makespan_s=10.0)
    assert s["requests"] == 100 and s["shots_per_s"] == 1000.0
    assert abs(s["p50_latency_s"] - 50.5) < 1e-9 and 99.0 < s["p99_latency_s"] <= 100.0


def test_small_requests_waiting_together_are_batched_in_order():
    """A slot that admits a batchable request also takes the batchable ones
    queued right behind it (arrival order, within the budget and max_batch);
    a non-batchable request ends the group; every request completes once."""
    lock = threading.Lock()
    groups = []

    def execute(req, slot, admit, fp):
        time.sleep(0.01)
        with lock:
            groups.append([req.rid])
        return Result(req.rid, 0, req.shots, req.arrival_s, admit, 0.0, fp)

    def execute_batch(reqs, slot, admit, fps):
        time.sleep(0.01)
        with lock:
            groups.append([r.rid for r in reqs])
        return [Result(r.rid, 0, r.shots, r.arrival_s, admit, 0.0, f) for r, f in zip(reqs, fps)]

    # shots < 100: batchable; the budget lets at most 5 small ones share a group
    sizes = [10, 20, 30, 500, 40, 50, 60, 70, 80, 90, 15, 700, 25]
    sch = Scheduler(slots=1, budget_bytes=1000, footprint=lambda r: r.shots, execute=execute,
                    execute_batch=execute_batch, batchable=lambda r: r.shots < 100, max_batch=4)
    res = sch.run(_reqs(sizes), realtime=False)
    assert sorted(r.rid for r in res) == list(range(len(sizes)))
    flat = [rid for g in groups for rid in g]
    assert flat == list(range(len(sizes)))  # one slot: FIFO order, no overtaking
    for g in groups:
        assert len(g) <= 4
        if len(g) > 1:
            assert all(sizes[r] < 100 for r in g)
            assert g == list(range(g[0], g[0] + len(g)))  # consecutive in the queue
    assert sch.batches >= 2 and sch.batched_requests >= 6
    assert sch.peak_in_use <= 1000
