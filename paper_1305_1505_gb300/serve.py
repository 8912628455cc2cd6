"""Request loop for collapse-time requests: continuous batching with
admission by device-memory footprint.

A request asks for the collapse times of one realisation (grid N, box L,
seed, radii).  The server keeps a FIFO queue; a request is admitted as soon
as a slot is free and its workspace (pin_footprint_bytes) fits in what is
left of the memory budget, so requests that arrive while others are running
start on their own streams and their work overlaps on the device.  Each
request's delta(k) and running-F state stay on the device from pin_set_ic to
the end of its radius loop; only F_max and the scale index come back.

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


class PinEngine:
    """Runs one request on the GPU: a plan on a stream of its own, the x/y
    tile widths the tuner chose for its grid size (pin_autotune keeps one
    choice per shape for the process; `warm` makes them before traffic
    arrives), delta(k) generated on the device from the request's seed
    (pin_set_ic_seed), the whole radius loop, results copied to the host."""

    def __init__(self, device=0, priority_from_n=0):
        """priority_from_n > 0: requests with N at or above it run on a
        high-priority stream (the device's block scheduler then serves their
        kernels first), the rest on normal ones."""
        import torch
        self.torch = torch
        self.device = device
        self.priority_from_n = int(priority_from_n)

    def warm(self, sizes, box_per_cell=2.0):
        """Loads the library and tunes the tile widths of each grid size on an
        idle device (a plan per size, timed alone, then freed)."""
        self.torch.cuda.set_device(self.device)
        out = {}
        for n in sizes:
            plan = pin.Plan(n, box_per_cell * n, [8.0, 4.0])
            try:
                out[int(n)] = plan.autotune(reps=3)
            finally:
                plan.close()
        return out

    def footprint(self, req):
        return pin.pin_footprint_bytes(pin.make_desc(req.n, req.box, req.radii))

    def run(self, req, timeout_s=None):
        torch = self.torch
        torch.cuda.set_device(self.device)
        high = self.priority_from_n > 0 and req.n >= self.priority_from_n
        stream = torch.cuda.Stream(priority=-1 if high else 0)
        plan = pin.Plan(req.n, req.box, req.radii, stream=stream)
        try:
            plan.autotune()  # the kept choice for this shape (timed once per process)
            n = req.n
            F = torch.empty((n, n, n), dtype=torch.float32, device="cuda")
            I = torch.empty((n, n, n), dtype=torch.int32, device="cuda")
            torch.cuda.current_stream().synchronize()
            pin.pin_set_ic_seed(plan.handle, req.seed)
            pin.pin_collapse_times(plan.handle, F.data_ptr(), I.data_ptr(), 1)
            st = pin.pin_sync(plan.handle, -1 if timeout_s is None else int(timeout_s * 1e9))
            if st == pin.PIN_ETIMEOUT:
                plan.sync()  # the device work cannot be cancelled: drain before freeing
                raise TimeoutError("device work exceeded the request deadline")
            pin._check(st, plan.handle)
            return F.cpu().numpy(), I.cpu().numpy()
        finally:
            plan.close()


class Server:
    """FIFO admission by memory footprint and slot count; one worker thread
    per admitted request."""

    def __init__(self, engine, budget_bytes, max_slots=4):
        self.engine = engine
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
                    if self.queue:
                        head = self.queue[0]
                        if self.running < self.max_slots and self.in_use + head.footprint <= self.budget:
                            break
                    self.lock.wait(0.01)
                if self._stop:
                    return
                req = self.queue.popleft()
                self.in_use += req.footprint
                self.running += 1
                self.peak_in_use = max(self.peak_in_use, self.in_use)
                self.peak_running = max(self.peak_running, self.running)
                req.t_admit = time.perf_counter()
                req.status = "running"
            threading.Thread(target=self._work, args=(req,), daemon=True).start()

    def _work(self, req):
        remaining = None
        if req.deadline is not None:
            remaining = max(0.0, req.deadline - (time.perf_counter() - req.arrival))
        try:
            res = self.engine.run(req, remaining)
            status, err = "done", None
        except TimeoutError as e:
            res, status, err = None, "timeout", str(e)
        except Exception as e:  # reported per request
            res, status, err = None, "failed", "%s: %s" % (type(e).__name__, e)
        with self.lock:
            self.in_use -= req.footprint
            self.running -= 1
            self._finish(req, status, res, err)
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


def main():
    import torch
    ap = argparse.ArgumentParser(description="serve a Poisson stream of mixed collapse-time requests")
    ap.add_argument("--requests", type=int, default=120)
    ap.add_argument("--rate", type=float, default=2.0, help="mean arrivals per second")
    ap.add_argument("--stress-rate", type=float, default=0.0,
                    help="also replay the same mix at this rate (0: skip), to load the device")
    ap.add_argument("--seed", type=int, default=5)
    ap.add_argument("--slots", type=int, default=4)
    ap.add_argument("--budget-gb", type=float, default=0.0, help="0: 80%% of free device memory")
    ap.add_argument("--priority-from-n", type=int, default=0,
                    help="grid size from which requests run on a high-priority stream (0: none)")
    args = ap.parse_args()
    free, _ = torch.cuda.mem_get_info()
    budget = int(args.budget_gb * 2 ** 30) if args.budget_gb > 0 else int(0.8 * free)
    eng = PinEngine(priority_from_n=args.priority_from_n)
    tiles = eng.warm([64, 128, 256, 512])
    eng.run(Request(-1, 64, 128.0, 1, [8.0, 4.0]))  # warm up
    def measure(rate):
        stream = workload(args.requests, args.seed, rate)
        served, wall_s, srv = replay(lambda: Server(eng, budget, args.slots), stream)
        plain, wall_p, _ = replay(lambda: Server(eng, budget, 1), stream)
        return {"rate_per_s": rate,
                "served": dict(_stats(served, wall_s), slots=args.slots,
                               peak_running=srv.peak_running, budget_bytes=budget),
                "plain_one_at_a_time": _stats(plain, wall_p)}

    line = {"metric": "served collapse-time requests: latency p50/p99 and throughput",
            "workload": "%d requests, Poisson arrivals, N in {64,128,256,512} (.4/.3/.2/.1), "
                        "box 2 Mpc/h per cell, 20-40 radii 40->2 Mpc/h, seed %d"
                        % (args.requests, args.seed),
            "tiles": {str(k): list(v) for k, v in tiles.items()},
            "priority_from_n": args.priority_from_n,
            "nominal": measure(args.rate)}
    if args.stress_rate > 0:
        line["stress"] = measure(args.stress_rate)
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
