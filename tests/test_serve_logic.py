"""Scheduling logic of the request server on the CPU, with a fake engine:
memory-budget admission, slot limit, rejection, queue deadlines, failures."""
import threading
import time

import numpy as np

from paper_1305_1505_gb300 import serve


class FakeEngine:
    def __init__(self, dur=0.05, fail_ids=()):
        self.dur = dur
        self.fail_ids = set(fail_ids)
        self.lock = threading.Lock()
        self.active = 0
        self.peak = 0

    def footprint(self, req):
        return req.n * 1000

    def run(self, req, timeout_s=None):
        with self.lock:
            self.active += 1
            self.peak = max(self.peak, self.active)
        try:
            time.sleep(self.dur)
            if req.rid in self.fail_ids:
                raise RuntimeError("engine failure")
            return (req.n, req.seed)
        finally:
            with self.lock:
                self.active -= 1


def _req(i, n, deadline=None):
    return serve.Request(i, n, 2.0 * n, 100 + i, [4.0, 2.0], deadline_s=deadline)


def test_budget_and_slots_bound_concurrency():
    eng = FakeEngine(dur=0.05)
    srv = serve.Server(eng, budget_bytes=100_000, max_slots=3)
    reqs = [srv.submit(_req(i, 40)) for i in range(10)]  # 40 kB each: 2 fit the budget
    assert srv.drain(timeout=10)
    srv.close()
    assert all(r.status == "done" for r in reqs)
    assert srv.peak_in_use <= 100_000
    assert srv.peak_running == 2 and eng.peak == 2
    assert [r.result for r in reqs] == [(40, 100 + i) for i in range(10)]


def test_slot_limit():
    eng = FakeEngine(dur=0.05)
    srv = serve.Server(eng, budget_bytes=10 ** 9, max_slots=3)
    reqs = [srv.submit(_req(i, 8)) for i in range(9)]
    assert srv.drain(timeout=10)
    srv.close()
    assert srv.peak_running == 3 and all(r.status == "done" for r in reqs)


def test_over_budget_request_is_rejected_immediately():
    srv = serve.Server(FakeEngine(), budget_bytes=50_000, max_slots=2)
    r = srv.submit(_req(0, 64))
    assert r.status == "rejected" and "exceeds" in r.error
    ok = srv.submit(_req(1, 16))
    assert ok.wait(5) == "done"
    srv.close()


def test_queue_deadline():
    eng = FakeEngine(dur=0.3)
    srv = serve.Server(eng, budget_bytes=10 ** 9, max_slots=1)
    first = srv.submit(_req(0, 8))
    late = srv.submit(_req(1, 8, deadline=0.05))
    assert late.wait(5) == "timeout" and "queue" in late.error
    assert first.wait(5) == "done"
    srv.close()


def test_engine_failure_is_reported_and_slot_released():
    eng = FakeEngine(dur=0.01, fail_ids={1})
    srv = serve.Server(eng, budget_bytes=10 ** 9, max_slots=1)
    reqs = [srv.submit(_req(i, 8)) for i in range(3)]
    assert srv.drain(timeout=5)
    srv.close()
    assert [r.status for r in reqs] == ["done", "failed", "done"]
    assert "engine failure" in reqs[1].error
    assert srv.in_use == 0 and srv.running == 0


def test_workload_mix_is_seeded():
    a = serve.workload(200, seed=5)
    b = serve.workload(200, seed=5)
    assert [x[1:4] for x in a] == [x[1:4] for x in b]
    ns = np.array([x[1] for x in a])
    assert set(ns) <= {64, 128, 256, 512}
    assert abs((ns == 64).mean() - 0.4) < 0.1
    assert all(20 <= x[4].size <= 40 for x in a)
    t = np.array([x[0] for x in a])
    assert np.all(np.diff(t) >= 0) and 50 < t[-1] < 150  # ~2 arrivals per second


def test_close_cancels_queued_requests_and_lets_running_ones_finish():
    eng = FakeEngine(dur=0.3)
    srv = serve.Server(eng, budget_bytes=10 ** 9, max_slots=1)
    reqs = [srv.submit(_req(i, 64)) for i in range(4)]
    time.sleep(0.05)  # the first is admitted, the rest wait for the slot
    srv.close()
    for r in reqs[1:]:
        assert r.wait(timeout=2.0) == "cancelled"
    assert reqs[0].wait(timeout=2.0) == "done"
    assert reqs[0].result == (64, 100)


def test_large_requests_do_not_share_the_device_and_do_not_block_small_ones():
    """At most max_big large requests (N >= big_n) run at once; a small
    request queued behind a held large one is admitted meanwhile."""
    eng = FakeEngine(dur=0.1)
    running_big, peak_big = [0], [0]
    lock = threading.Lock()
    orig = eng.run

    def run(req, timeout_s=None):
        big = req.n >= 512
        with lock:
            running_big[0] += big
            peak_big[0] = max(peak_big[0], running_big[0])
        try:
            return orig(req, timeout_s)
        finally:
            with lock:
                running_big[0] -= big

    eng.run = run
    srv = serve.Server(eng, budget_bytes=10 ** 9, max_slots=4, big_n=512, max_big=1)
    reqs = [srv.submit(_req(0, 512)), srv.submit(_req(1, 512)), srv.submit(_req(2, 64))]
    time.sleep(0.05)
    # the second large request waits; the small one behind it already runs
    assert reqs[1].status == "queued" and reqs[2].status in ("running", "done")
    assert srv.drain(timeout=5)
    srv.close()
    assert all(r.status == "done" for r in reqs)
    assert peak_big[0] == 1
    assert reqs[2].t_done < reqs[1].t_done
