"""Request loop for collapse-time requests: continuous batching with
admission by device-memory footprint.

A request asks for the collapse times of one realisation (grid N, box L,
seed, radii).  The server keeps a FIFO queue; a request is admitted as soon
as a slot is free and its workspace (pin_footprint_bytes) fits in what is
left of the memory budget, so requests that arrive while others are running
start on their own streams and their work overlaps on the device.  The
engine runs each request on a pooled plan of its grid size (no device
allocation, free or graph capture per request once the pool is warm).  Each
request's delta(k) and running-F state stay on the device from its seeded
generation to the end of its radius loop; only F_max and the scale index come
back, into page-locked host memory.

Failures are reported per request, never by a device trap:
  rejected  its footprint exceeds the whole budget (PIN_EBUSY semantics);
  cancelled the server was closed while it waited in the queue;
  timeout   it waited in the queue, or its device work ran, past its deadline
            (the device work cannot be cancelled: its slot and memory are held
            until it drains, then released).

The engine is a small interface (footprint, run), so the scheduling logic is
tested on the CPU with a fake engine and on the GPU with PinEngine.
"""
import argparse
import collections
import json
import threading
import time

import numpy as np

from . import pin


class Request:
    __slots__ = ("rid", "n", "box", "seed", "radii", "arrival", "deadline", "t_admit", "t_done",
                 "status", "result", "error", "footprint", "_event")

    def __init__(self, rid, n, box, seed, radii, deadline_s=None):
        self.rid = rid
        self.n = int(n)
        self.box = float(box)
        self.seed = int(seed)
        self.radii = np.ascontiguousarray(radii, dtype=np.float64)
        self.arrival = None
        self.deadline = deadline_s
        self.t_admit = None
        self.t_done = None
        self.status = "queued"
        self.result = None
        self.error = None
        self.footprint = 0
        self._event = threading.Event()

    def wait(self, timeout=None):
        self._event.wait(timeout)
        return self.status

    @property
    def latency(self):
        return None if self.t_done is None else self.t_done - self.arrival

    @property
    def updates(self):
        return self.n ** 3 * self.radii.size


class _Slot:
    """A pooled plan of one grid size with everything a request needs: its
    stream, device outputs and page-locked host outputs."""
    __slots__ = ("key", "plan", "stream", "F", "I", "hF", "hI")


class PinEngine:
    """Runs requests on the GPU from a pool of plans per grid size (and box).

    A request takes an idle plan of its size (a new one is made only when none
    is idle), switches it to its radii (pin_set_radii: the workspace stays, the
    graph of a radius count is captured once), generates its delta(k) on the
    device from its seed (pin_set_ic_seed), runs the whole radius loop and
    copies F_max and the index into the plan's page-locked host buffers, all on
    the plan's stream.  After warm-up no request allocates or frees device
    memory, so no request pays a cudaMalloc, the device-wide synchronisation of
    a cudaFree, or a graph capture.  The result arrays are views of the plan's
    host buffers: the plan returns to the pool when the request is released
    (Request.release, called by the server once the result has been handed on,
    or by the caller when it keeps the request)."""

    def __init__(self, device=0, priority_from_n=0, pool_per_size=4):
        """priority_from_n > 0: plans for N at or above it run on high-priority
        streams (the device's block scheduler then serves their kernels first),
        the rest on normal ones.  pool_per_size: idle plans kept per size."""
        import torch
        self.torch = torch
        self.device = device
        self.priority_from_n = int(priority_from_n)
        self.pool_per_size = int(pool_per_size)
        self.pool = collections.defaultdict(list)
        self.lock = threading.Lock()
        self.plans_made = 0

    def _make(self, n, box):
        torch = self.torch
        torch.cuda.set_device(self.device)
        high = self.priority_from_n > 0 and n >= self.priority_from_n
        s = _Slot()
        s.key = (int(n), float(box))
        s.stream = torch.cuda.Stream(priority=-1 if high else 0)
        s.plan = pin.Plan(n, box, [8.0, 4.0], stream=s.stream)
        s.plan.autotune()  # the kept choice for this shape (timed once per process)
        s.F = torch.empty((n, n, n), dtype=torch.float32, device="cuda")
        s.I = torch.empty((n, n, n), dtype=torch.int32, device="cuda")
        s.hF = torch.empty((n, n, n), dtype=torch.float32).pin_memory()
        s.hI = torch.empty((n, n, n), dtype=torch.int32).pin_memory()
        torch.cuda.synchronize()
        with self.lock:
            self.plans_made += 1
        return s

    def warm(self, sizes, box_per_cell=2.0, per_size=1):
        """Loads the library, tunes the tile widths and radix schedules of
        each grid size on an idle device and fills the pool with per_size plans
        of each size.  Returns, per size, ((tc_x, tc_y), (radix_x, radix_y))."""
        out = {}
        for n in sizes:
            slots = [self._make(n, box_per_cell * n) for _ in range(per_size)]
            out[int(n)] = (slots[0].plan.tiles(), slots[0].plan.radix())
            for s in slots:
                self._release(s)
        return out

    def _acquire(self, n, box):
        with self.lock:
            idle = self.pool[(int(n), float(box))]
            if idle:
                return idle.pop()
        return self._make(n, box)

    def _release(self, slot):
        with self.lock:
            idle = self.pool[slot.key]
            if len(idle) < self.pool_per_size:
                idle.append(slot)
                return
        slot.plan.close()

    def close(self):
        with self.lock:
            slots = [s for v in self.pool.values() for s in v]
            self.pool.clear()
        for s in slots:
            s.plan.close()

    def footprint(self, req):
        return pin.pin_footprint_bytes(pin.make_desc(req.n, req.box, req.radii))

    def run(self, req, timeout_s=None):
        """Returns (F_max, scale_idx, release): numpy views of the plan's host
        buffers and the callable that hands the plan back to the pool."""
        torch = self.torch
        torch.cuda.set_device(self.device)
        slot = self._acquire(req.n, req.box)
        ok = False
        try:
            plan = slot.plan
            plan.set_radii(req.radii)
            pin.pin_set_ic_seed(plan.handle, req.seed)
            pin.pin_collapse_times(plan.handle, slot.F.data_ptr(), slot.I.data_ptr(), 1)
            with torch.cuda.stream(slot.stream):  # after the radius loop, on the plan's stream
                slot.hF.copy_(slot.F, non_blocking=True)
                slot.hI.copy_(slot.I, non_blocking=True)
            st = pin.pin_sync(plan.handle, -1 if timeout_s is None else int(timeout_s * 1e9))
            if st == pin.PIN_ETIMEOUT:
                plan.sync()  # the device work cannot be cancelled: drain before reuse
                raise TimeoutError("device work exceeded the request deadline")
            pin._check(st, plan.handle)
            ok = True
            return slot.hF.numpy(), slot.hI.numpy(), (lambda: self._release(slot))
        finally:
            if not ok:
                self._release(slot)


class Server:
    """FIFO admission by memory footprint and slot count; one worker thread
    per admitted request.  Large requests (N >= big_n) are admitted at most
    max_big at a time: two of them sharing the device would both take about
    twice as long, which sets the latency tail, while small requests cost the
    device little and overlap freely (and do not wait behind a large one)."""

    def __init__(self, engine, budget_bytes, max_slots=4, keep_results=True, big_n=512, max_big=1):
        """keep_results: copy each result into arrays of the request (False:
        drop it; latency is measured to the result's arrival in host memory
        either way).  big_n / max_big: the large-request limit (max_big 0:
        none)."""
        self.engine = engine
        self.keep_results = bool(keep_results)
        self.big_n = int(big_n)
        self.max_big = int(max_big)
        self.running_big = 0
        self.budget = int(budget_bytes)
        self.max_slots = int(max_slots)
        self.queue = collections.deque()
        self.lock = threading.Condition()
        self.in_use = 0
        self.running = 0
        self.peak_in_use = 0
        self.peak_running = 0
        self.done = []
        self._stop = False
        self._sched = threading.Thread(target=self._schedule, daemon=True)
        self._sched.start()

    def _is_big(self, req):
        return self.max_big > 0 and req.n >= self.big_n

    def submit(self, req, now=None):
        req.arrival = time.perf_counter() if now is None else now
        req.footprint = self.engine.footprint(req)
        with self.lock:
            if req.footprint > self.budget:
                self._finish(req, "rejected", error="footprint %d B exceeds the budget %d B"
                             % (req.footprint, self.budget))
                return req
            self.queue.append(req)
            self.lock.notify_all()
        return req

    def _finish(self, req, status, result=None, error=None):
        req.status = status
        req.result = result
        req.error = error
        req.t_done = time.perf_counter()
        self.done.append(req)
        req._event.set()

    def _schedule(self):
        while True:
            with self.lock:
                while not self._stop:
                    now = time.perf_counter()
                    # drop queued requests whose deadline passed
                    while self.queue and self.queue[0].deadline is not None and \
                            now - self.queue[0].arrival > self.queue[0].deadline:
                        self._finish(self.queue.popleft(), "timeout", error="deadline passed in the queue")
                    # FIFO, except that a large request held by the large-request
                    # limit lets the requests behind it pass; the first one not
                    # so held is admitted when its memory fits, else everyone
                    # waits (no overtaking on memory, so none starves)
                    pick = None
                    if self.running < self.max_slots:
                        for i, r in enumerate(self.queue):
                            if self._is_big(r) and self.running_big >= self.max_big:
                                continue
                            if self.in_use + r.footprint <= self.budget:
                                pick = i
                            break
                    if pick is not None:
                        break
                    self.lock.wait(0.01)
                if self._stop:
                    return
                req = self.queue[pick]
                del self.queue[pick]
                self.in_use += req.footprint
                self.running += 1
                self.running_big += 1 if self._is_big(req) else 0
                self.peak_in_use = max(self.peak_in_use, self.in_use)
                self.peak_running = max(self.peak_running, self.running)
                req.t_admit = time.perf_counter()
                req.status = "running"
            threading.Thread(target=self._work, args=(req,), daemon=True).start()

    def _work(self, req):
        remaining = None
        if req.deadline is not None:
            remaining = max(0.0, req.deadline - (time.perf_counter() - req.arrival))
        release = None
        t_done = None
        try:
            res = self.engine.run(req, remaining)
            t_done = time.perf_counter()
            if isinstance(res, tuple) and len(res) == 3 and callable(res[2]):
                res, release = res[:2], res[2]  # views of a pooled plan's buffers
                res = tuple(np.array(a) for a in res) if self.keep_results else None
            status, err = "done", None
        except TimeoutError as e:
            res, status, err = None, "timeout", str(e)
        except Exception as e:  # reported per request
            res, status, err = None, "failed", "%s: %s" % (type(e).__name__, e)
        finally:
            if release is not None:
                release()
        with self.lock:
            self.in_use -= req.footprint
            self.running -= 1
            self.running_big -= 1 if self._is_big(req) else 0
            self._finish(req, status, res, err)
            if t_done is not None:
                req.t_done = t_done
            self.lock.notify_all()

    def drain(self, timeout=None):
        t0 = time.perf_counter()
        while True:
            with self.lock:
                if not self.queue and self.running == 0:
                    return True
            if timeout is not None and time.perf_counter() - t0 > timeout:
                return False
            time.sleep(0.005)

    def close(self):
        """Stops admitting: requests still queued are finished as "cancelled"
        (their waiters wake up); admitted ones run to completion."""
        with self.lock:
            self._stop = True
            while self.queue:
                self._finish(self.queue.popleft(), "cancelled", error="server closed before admission")
            self.lock.notify_all()
        self._sched.join(timeout=5)


def workload(count, seed=5, rate=2.0):
    """Mixed request stream: N in {64,128,256,512} (weights .4/.3/.2/.1),
    box 2 Mpc/h per cell, 20..40 radii log-spaced 40 -> 2 Mpc/h, seeds and
    Poisson arrival times from a seeded generator."""
    from . import ic
    rng = np.random.default_rng(seed)
    ns = rng.choice([64, 128, 256, 512], size=count, p=[0.4, 0.3, 0.2, 0.1])
    ss = rng.integers(20, 41, size=count)
    gaps = rng.exponential(1.0 / rate, size=count)
    out = []
    for i in range(count):
        n = int(ns[i])
        radii = ic.log_radii(2.0, 40.0, int(ss[i]))
        out.append((float(np.sum(gaps[: i + 1])), n, 2.0 * n, int(ic.splitmix64(seed + i) >> 33), radii))
    return out


def _stats(reqs, wall):
    lat = np.array([r.latency for r in reqs if r.status == "done"])
    upd = sum(r.updates for r in reqs if r.status == "done")
    return {"completed": int(lat.size), "p50_s": float(np.percentile(lat, 50)) if lat.size else None,
            "p99_s": float(np.percentile(lat, 99)) if lat.size else None,
            "mean_s": float(lat.mean()) if lat.size else None,
            "requests_per_s": lat.size / wall, "updates_per_s": upd / wall, "wall_s": wall}


def replay(server_factory, stream, realtime=True):
    """Submits the stream at its arrival times; returns (requests, wall time)."""
    srv = server_factory()
    t0 = time.perf_counter()
    reqs = []
    for i, (t_arr, n, box, seed, radii) in enumerate(stream):
        if realtime:
            delay = t0 + t_arr - time.perf_counter()
            if delay > 0:
                time.sleep(delay)
        reqs.append(srv.submit(Request(i, n, box, seed, radii)))
    srv.drain()
    wall = time.perf_counter() - t0
    srv.close()
    return reqs, wall, srv


def measure_serving(requests=600, rate=2.0, seed=5, slots=4, budget_bytes=0, priority_from_n=0,
                    stress_rate=0.0):
    """The mixed request stream served with `slots` concurrent requests and
    one at a time, on the same engine and plan pool; latency p50/p99 and
    throughput of both (a dict).  budget_bytes 0: 80 % of free device memory."""
    import torch
    free, _ = torch.cuda.mem_get_info()
    budget = int(budget_bytes) if budget_bytes > 0 else int(0.8 * free)
    eng = PinEngine(priority_from_n=priority_from_n, pool_per_size=slots)
    sizes = [64, 128, 256, 512]
    tiles = eng.warm(sizes, per_size=slots)
    for n in sizes:  # first launch of each size, outside the measurement
        _, _, rel = eng.run(Request(-1, n, 2.0 * n, 1, [8.0, 4.0]))
        rel()
    made0 = eng.plans_made

    def one(rate_):
        stream = workload(requests, seed, rate_)
        served, wall_s, srv = replay(lambda: Server(eng, budget, slots, keep_results=False), stream)
        plain, wall_p, _ = replay(lambda: Server(eng, budget, 1, keep_results=False), stream)
        return {"rate_per_s": rate_,
                "served": dict(_stats(served, wall_s), slots=slots, peak_running=srv.peak_running,
                               budget_bytes=budget),
                "plain_one_at_a_time": _stats(plain, wall_p)}

    out = {"metric": "served collapse-time requests: latency p50/p99 and throughput",
           "workload": "%d requests, Poisson arrivals (mean %g/s), N in {64,128,256,512} (.4/.3/.2/.1), "
                       "box 2 Mpc/h per cell, 20-40 radii 40->2 Mpc/h, seed %d" % (requests, rate, seed),
           "tiles": {str(k): {"tiles": list(v[0]), "radix": list(v[1])} for k, v in tiles.items()},
           "priority_from_n": priority_from_n,
           "nominal": one(rate)}
    if stress_rate > 0:
        out["stress"] = one(stress_rate)
    out["plans_made_during_traffic"] = eng.plans_made - made0
    eng.close()
    return out


def main():
    ap = argparse.ArgumentParser(description="serve a Poisson stream of mixed collapse-time requests")
    ap.add_argument("--requests", type=int, default=600)
    ap.add_argument("--rate", type=float, default=2.0, help="mean arrivals per second")
    ap.add_argument("--stress-rate", type=float, default=0.0,
                    help="also replay the same mix at this rate (0: skip), to load the device")
    ap.add_argument("--seed", type=int, default=5)
    ap.add_argument("--slots", type=int, default=4)
    ap.add_argument("--budget-gb", type=float, default=0.0, help="0: 80%% of free device memory")
    ap.add_argument("--priority-from-n", type=int, default=0,
                    help="grid size from which requests run on a high-priority stream (0: none)")
    args = ap.parse_args()
    line = measure_serving(args.requests, args.rate, args.seed, args.slots, int(args.budget_gb * 2 ** 30),
                           args.priority_from_n, args.stress_rate)
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
