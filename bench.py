"""Benchmark of the collapse-time path: collapse updates/s (particles x radii).

Workload (default): 768^3 grid, box 3072 Mpc/h, seeded Gaussian field with
P(k) = A k^0.96 T_BBKS(k/0.21)^2, sigma8 = 0.8, seed 3, 40 Gaussian radii
log-spaced from 120 down to 4 Mpc/h.  One step = one pin_collapse_times call
(all radii: filter, inverse FFTs of the six Hessian components, eigenvalues,
collapse time, running maximum) with delta(k) resident on the device.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

N > 1 runs N independent replicas (one per rank, launched by torchrun); the
path has no data exchange, so value = all ranks' updates / max-over-ranks time.
--impl reference times the FP64 CPU oracle on the host cores on a bounded
sample of the same workload (the paper has no GPU implementation to run).
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = dict(n=768, box=3072.0, seed=3, nscales=40, r_min=4.0, r_max=120.0)
# bounded CPU sample: same 4 Mpc/h cells and spectrum on a 128^3 grid, six of
# the forty radii (every seventh, largest first)
CPU_SAMPLE = dict(n=128, box=512.0, seed=3, every=7)
METRIC = "collapse updates/s (particles x scales) at 768^3"
UNIT = "updates/s"


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return d["hbm_gbs"], "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.lines = []
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()
                out = ""
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in getattr(self, "lines", []):
            parts = [x.strip() for x in l.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower() in ("active", "1", "yes"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def algorithmic_bytes(n, fused, velocities):
    """Bytes each pass must move per launch (one launch per radius).
    A half-spectrum is H = N^2 (N/2+1) complex64 values (8H bytes, ~4 B per
    particle).  x: read Phi0, write 3 spectra.  y: read 3, write 6 (+3 psi
    spectra with velocities).  z: read those spectra; split layout: write 3
    eigenvalue floats per particle (+3 psi floats), then the root pass reads
    them; the running-maximum state is an F_max read plus F_max and index
    writes, 12 B per particle (writes are an upper bound: only where F rises),
    +12 B for the velocity state (+12 B psi read in the split layout)."""
    H = n * n * (n // 2 + 1)
    N3 = n ** 3
    v = 1 if velocities else 0
    state = 12 * N3 + 12 * N3 * v
    alg = {"x": 4 * 8 * H, "y": (9 + 3 * v) * 8 * H}
    if fused:
        alg["z"] = (6 + 3 * v) * 8 * H + state
        alg["redo"] = 0
    else:
        alg["z"] = (6 + 3 * v) * 8 * H + 12 * N3 + 12 * N3 * v
        alg["roots"] = 12 * N3 + 12 * N3 * v + state
    return alg


# Counters of the dominant kernel, valid only while the kernel sources hash to
# the recorded value (otherwise reported as null): DRAM read + write bytes and
# warp instructions per particle and launch, averaged over the 40 launches of
# one step of the 384^3 x 40 workload (the same 4 Mpc/h cells and radii; a
# small case of 2.7 GB on the device, one ncu pass), scaled to a launch of the
# benchmark by its particle count.  The 768-point line transform has one more
# radix-2 level than the 384-point one, so the instruction count is a slight
# underestimate at 768^3.
TRAFFIC_SOURCES = ["kernels.cu", "kernels_v1.cu", "passes_xy.cuh", "kernels.cuh", "fft.cuh", "packed.cuh",
                   "collapse.cuh", "collapse_x2.cuh", "pin.cu"]
MEASURED_TRAFFIC = {
    # profiles/z_pass_instruction_mix_384.md
    ("k_pass_z", 768, False): {"sources": "3f2b757b0f7242b0", "bytes_per_particle": 30.239, "warp_inst_per_particle": 9.6018,
                               "measured_at": "384^3 x 40, the 40 launches of one step, scaled by particles"},
}


def code_text(src):
    """C/CUDA source without comments and with whitespace runs collapsed, so
    that a recorded measurement survives edits of comments only."""
    import re
    src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)
    src = re.sub(r"//[^\n]*", " ", src)
    return " ".join(src.split())


def sources_digest(read=None):
    """Digest of the code (not the comments) of the kernel sources;
    read(name) -> text overrides reading the working tree."""
    import hashlib
    h = hashlib.sha256()
    for f in TRAFFIC_SOURCES:
        if read is None:
            with open(os.path.join(ROOT, "paper_1305_1505_gb300", "csrc", f)) as fh:
                text = fh.read()
        else:
            text = read(f)
        h.update(code_text(text).encode())
    return h.hexdigest()[:16]


def measured_record(kernel, n, velocities):
    rec = MEASURED_TRAFFIC.get((kernel, n, bool(velocities)))
    if rec is None or rec["sources"] != sources_digest():
        return None
    return rec


def measured_traffic(kernel, n, nscales, velocities):
    rec = measured_record(kernel, n, velocities)
    return None if rec is None else rec["bytes_per_particle"] * n ** 3


# Issue roof of the SMs: 152 SMs x 4 warp schedulers x 1 warp instruction per
# cycle at the sampled maximum SM clock (2070 MHz on GB300).
SMS, SCHEDULERS = 152, 4


def roofline(pass_name, ms_per_launch, n, velocities, fused, hbm_achieved, hbm_peak, peak_kind, clocks, passes):
    """Roofline object of the dominant kernel.  HBM-bound passes report
    algorithmic GB/s against the measured copy bandwidth.  The fused z pass
    is bound by instruction issue: when its warp-instruction count per launch
    was measured on the current kernel sources (MEASURED_TRAFFIC), it reports
    warp instructions per second against the issue roof (SMS x SCHEDULERS x
    the sampled maximum SM clock), with its HBM fraction alongside."""
    kname = ("k_pass_" if pass_name in "xyz" else "k_") + pass_name
    rec = measured_record(kname, n, velocities)
    traffic = None if rec is None else rec["bytes_per_particle"] * n ** 3
    hbm = {"bound": "hbm", "kernel": kname, "achieved": hbm_achieved, "peak": hbm_peak,
           "peak_kind": peak_kind, "unit": "GB/s", "frac": hbm_achieved / hbm_peak,
           "traffic": traffic, "passes": passes}
    if rec is None or not fused or kname != "k_pass_z" or not rec.get("warp_inst_per_particle"):
        return hbm
    mhz = (clocks or {}).get("sm_max_mhz") or 2070.0
    peak = SMS * SCHEDULERS * mhz * 1e6 / 1e9
    achieved = rec["warp_inst_per_particle"] * n ** 3 / (ms_per_launch / 1e3) / 1e9
    return {"bound": "alu", "kernel": kname, "achieved": achieved, "peak": peak,
            "peak_kind": "derived: %d SMs x %d schedulers x 1 warp instruction/cycle x %.0f MHz"
                         % (SMS, SCHEDULERS, mhz),
            "unit": "Gwarp-inst/s", "frac": achieved / peak, "traffic": traffic,
            "counters_measured_at": rec.get("measured_at"),
            "hbm_frac": hbm_achieved / hbm_peak, "hbm_peak_kind": peak_kind, "passes": passes}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def replica_value(local_s, units_per_rank, world_size, device=None):
    """Replicas: the slowest rank's time and all ranks' units over it.

    Each rank processes its own realisation (no data exchange); the only
    collective is this max over ranks of the timed duration.  Returns
    (max_seconds, units_per_second_whole_job)."""
    import torch
    import torch.distributed as dist
    t = local_s
    if world_size > 1:
        x = torch.tensor([float(local_s)], dtype=torch.float64, device=device)
        dist.all_reduce(x, op=dist.ReduceOp.MAX)
        t = float(x.item())
    return t, units_per_rank * world_size / t


def cpu_baseline(nscales_total):
    """FP64 oracle, as it stands, on the bounded sample; updates/s and cores."""
    import oracle
    from paper_1305_1505_gb300 import ic
    s = CPU_SAMPLE
    radii = ic.log_radii(WORKLOAD["r_min"], WORKLOAD["r_max"], nscales_total)[::s["every"]]
    d = ic.delta_k(s["n"], s["box"], s["seed"], dtype=np.complex64).astype(np.complex128)
    oracle.lib()
    t0 = time.perf_counter()
    oracle.collapse_times(d, s["box"], radii)
    dt = time.perf_counter() - t0
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return {"value": s["n"] ** 3 * radii.size / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": "%d^3 grid, box %.0f Mpc/h (the same 4 Mpc/h cells), seed %d, %d of the %d radii"
                      " (every %dth), FP64, %.1f s" % (s["n"], s["box"], s["seed"], radii.size,
                                                       nscales_total, s["every"], dt)}


# The smaller single-realisation workloads: 64^3 / 100 Mpc/h, seed 1, 20 radii
# 15 -> 1.5625 Mpc/h (one cell), and 256^3 / 512 Mpc/h, seed 2, 30 radii
# 40 -> 2 Mpc/h (one cell); the oracle's sample for each (every radius of the
# small one, every tenth radius of the larger one).
CONFIGS = {
    "config1": dict(n=64, box=100.0, seed=1, nscales=20, r_min=100.0 / 64, r_max=15.0, every=1),
    "config2": dict(n=256, box=512.0, seed=2, nscales=30, r_min=2.0, r_max=40.0, every=10),
}


def measure_config(c, steps, warmup, tune=True):
    """Device-timed collapse updates/s of one workload (delta(k) resident),
    K steps back to back after the warm-up, and the whole step's
    algorithmic bytes over its time."""
    import torch
    from paper_1305_1505_gb300 import ic, pin
    n, S = c["n"], c["nscales"]
    radii = ic.log_radii(c["r_min"], c["r_max"], S)
    stream = torch.cuda.Stream()
    plan = pin.Plan(n, c["box"], radii, stream=stream)
    plan.set_ic(torch.from_numpy(ic.delta_k(n, c["box"], c["seed"], dtype=np.complex64)).cuda())
    tiles = plan.autotune(reps=5) if tune else plan.tiles()
    F = torch.empty((n, n, n), dtype=torch.float32, device="cuda")
    I = torch.empty((n, n, n), dtype=torch.int32, device="cuda")
    for _ in range(warmup):
        pin.pin_collapse_times(plan.handle, F.data_ptr(), I.data_ptr(), 1)
    plan.sync()
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
    torch.cuda.synchronize()
    evs[0].record(stream)
    for i in range(steps):
        pin.pin_collapse_times(plan.handle, F.data_ptr(), I.data_ptr(), 1)
        evs[i + 1].record(stream)
    torch.cuda.synchronize()
    ms = evs[0].elapsed_time(evs[-1]) / steps
    fused = pin.pin_kernels_per_call(plan.handle) == 4 * S
    alg = algorithmic_bytes(n, fused, False)
    peak, peak_kind = _peaks()
    step_bytes = S * sum(alg.values())
    out = {"workload": "%d^3 grid, box %.0f Mpc/h, seed %d, %d radii %.4g->%.4g Mpc/h (log)"
                       % (n, c["box"], c["seed"], S, c["r_max"], c["r_min"]),
           "value": n ** 3 * S / (ms / 1e3), "unit": UNIT, "ms_per_step": ms,
           "best_ms_per_step": min(evs[i].elapsed_time(evs[i + 1]) for i in range(steps)),
           "tiles": {"x": tiles[0], "y": tiles[1], "radix_x": plan.radix()[0], "radix_y": plan.radix()[1]},
           "step_alg_bytes_per_update": step_bytes / (n ** 3 * S),
           "step_hbm_frac": step_bytes / (ms / 1e3) / 1e9 / peak, "hbm_peak_kind": peak_kind,
           "gpu_launches": int(steps * pin.pin_kernels_per_call(plan.handle))}
    plan.close()
    return out


def config_cpu_baseline(c):
    """The oracle, as it stands, on a sample of the workload's radii."""
    import oracle
    from paper_1305_1505_gb300 import ic
    radii = ic.log_radii(c["r_min"], c["r_max"], c["nscales"])[::c["every"]]
    d = ic.delta_k(c["n"], c["box"], c["seed"], dtype=np.complex64).astype(np.complex128)
    oracle.lib()
    t0 = time.perf_counter()
    oracle.collapse_times(d, c["box"], radii)
    dt = time.perf_counter() - t0
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return {"value": c["n"] ** 3 * radii.size / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": "the same %d^3 field, %d of the %d radii (every %dth), FP64, %.1f s"
                      % (c["n"], radii.size, c["nscales"], c["every"], dt)}


def run_config(args, name):
    """One JSON line for a smaller workload, with the oracle beside it."""
    c = CONFIGS[name]
    m = measure_config(c, args.steps, args.warmup, tune=not args.no_tune)
    import torch
    with ClockSampler(torch.cuda.current_device()) as clk:
        pass
    line = {"metric": "collapse updates/s (particles x scales) at %d^3" % c["n"], "value": m["value"],
            "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": m["ms_per_step"], "best_ms_per_step": m["best_ms_per_step"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic", "config": {"workload": m["workload"], "tiles": m["tiles"]},
            "roofline": {"bound": "hbm", "kernel": "whole radius loop", "unit": "GB/s",
                         "achieved": m["step_hbm_frac"] * _peaks()[0], "peak": _peaks()[0],
                         "peak_kind": m["hbm_peak_kind"], "frac": m["step_hbm_frac"], "traffic": None,
                         "alg_bytes_per_update": m["step_alg_bytes_per_update"]},
            "cpu_baseline": None if args.no_cpu else config_cpu_baseline(c),
            "gpu_launches": m["gpu_launches"]}
    print(json.dumps(line), flush=True)
    return 0


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    w = WORKLOAD
    vals, secs = [], []
    cb = None
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        cb = cpu_baseline(w["nscales"])
        if i >= args.warmup:
            vals.append(cb["value"])
            secs.append(time.perf_counter() - t0)
    v = statistics.mean(vals)
    # a step of the full 768^3 x 40 workload would take this long at the
    # sampled rate; each timed step ran the bounded sample only
    ms = w["n"] ** 3 * w["nscales"] / v * 1e3
    cb["value"] = v
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "ms_per_step_extrapolated": True,
            "sample_ms_per_step": 1e3 * statistics.mean(secs),
            "extrapolation": "ms_per_step = 768^3 x 40 updates / the sampled updates/s; each step timed "
                             "the oracle on the bounded sample named in cpu_baseline",
            "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": _config(WORKLOAD),
            "cpu_baseline": cb,
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def _config(w):
    return {"workload": "%d^3 grid, box %.0f Mpc/h, seed %d, %d radii %.0f->%.0f Mpc/h (log), "
                        "BBKS Gamma=0.21 n=0.96 sigma8=0.8"
                        % (w["n"], w["box"], w["seed"], w["nscales"], w["r_max"], w["r_min"]),
            "grid": w["n"], "box_mpc_h": w["box"], "nscales": w["nscales"],
            "parallelism": "replicas",
            "l2": "inputs larger than L2 (delta(k) 1.8 GB, per-pass spectra 5.5-11 GB)"}


def run_ours(args):
    import torch
    import torch.distributed as dist

    from paper_1305_1505_gb300 import ic, pin

    ws, rank, local = _dist()
    if ws > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    w = dict(WORKLOAD)
    if args.grid:
        # smaller grid with the same 4 Mpc/h cells (profiling captures)
        w["n"], w["box"] = args.grid, 4.0 * args.grid
    if args.nscales:
        w["nscales"] = args.nscales
    n, S = w["n"], w["nscales"]
    radii = ic.log_radii(w["r_min"], w["r_max"], S)
    stream = torch.cuda.Stream()
    d32 = ic.delta_k(n, w["box"], w["seed"] + 1000 * rank if ws > 1 else w["seed"], dtype=np.complex64)
    if not args.no_e2e:
        # pinned host buffers of the end-to-end leg, allocated before the
        # plan and reused by every step
        hd = torch.from_numpy(d32).pin_memory()
        hF = torch.empty((n, n, n), dtype=torch.float32).pin_memory()
        hI = torch.empty((n, n, n), dtype=torch.int32).pin_memory()
    plan = pin.Plan(n, w["box"], radii, stream=stream, velocities=args.velocities)
    dk = torch.from_numpy(d32).cuda()
    plan.set_ic(dk)
    # x/y tile widths timed on this plan, outside the timed region
    if args.schedule:
        pin.pin_set_schedule(plan.handle, args.schedule)
    if args.radix:
        rx, ry = (int(v) for v in args.radix.split(","))
        plan.set_radix(rx, ry)
    if args.tiles:
        tx, ty = (int(v) for v in args.tiles.split(","))
        plan.set_tiles(tx, ty)
    tiles = plan.tiles() if (args.no_tune or args.tiles or args.radix) else plan.autotune(reps=5)
    F = torch.empty((n, n, n), dtype=torch.float32, device="cuda")
    I = torch.empty((n, n, n), dtype=torch.int32, device="cuda")
    pin.pin_profile(plan.handle, 1)

    def step():
        pin.pin_collapse_times(plan.handle, F.data_ptr(), I.data_ptr(), 1)

    for _ in range(args.warmup):
        step()
    plan.sync()

    def barrier():
        if ws > 1:
            dist.barrier()

    # K steps back to back on the plan's stream, no host synchronisation
    # between them; an event between steps gives the best single step
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    barrier()
    torch.cuda.synchronize()
    with ClockSampler(torch.cuda.current_device()) as clk:
        evs[0].record(stream)
        for i in range(args.steps):
            step()
            evs[i + 1].record(stream)
        torch.cuda.synchronize()
    barrier()
    # per-pass device times of the last timed step (event records inside its
    # graph, on the plan's stream), summed over its S radii
    pass_ms = np.array(pin.pin_pass_times(plan.handle))
    step_ms = [evs[i].elapsed_time(evs[i + 1]) for i in range(args.steps)]
    updates = n ** 3 * S
    total_s, _ = replica_value(evs[0].elapsed_time(evs[-1]) / 1e3, updates * args.steps, ws, "cuda")
    ms = total_s * 1e3 / args.steps
    value = updates * ws / (ms / 1e3)

    # end to end through the public API with host buffers: pinned delta(k) in,
    # F_max and scale index out, copies inside the timed region
    pin.pin_profile(plan.handle, 0)
    e2e_s = float("nan")
    e2e_parts = None
    if not args.no_e2e:
        e2e_steps = max(1, min(args.steps, 3))
        pin.pin_set_ic(plan.handle, hd.data_ptr(), pin.PIN_C64, 0)
        pin.pin_collapse_times(plan.handle, hF.data_ptr(), hI.data_ptr(), 0)  # warm graph
        barrier()
        t_ic, t_col = [], []
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            ta = time.perf_counter()
            pin.pin_set_ic(plan.handle, hd.data_ptr(), pin.PIN_C64, 0)  # H2D, Phi0, sync
            tb = time.perf_counter()
            pin.pin_collapse_times(plan.handle, hF.data_ptr(), hI.data_ptr(), 0)  # graph, D2H, sync
            tc = time.perf_counter()
            t_ic.append(tb - ta)
            t_col.append(tc - tb)
        e2e_s = (time.perf_counter() - t0) / e2e_steps
        ic_ms, col_ms = 1e3 * float(np.mean(t_ic)), 1e3 * float(np.mean(t_col))
        d2h_ms = max(col_ms - ms, 1e-6)  # the graph itself takes ms (device-timed above)
        # the same pinned buffers copied by torch in this process, for comparison
        dev_in = torch.empty(hd.shape, dtype=hd.dtype, device="cuda")
        torch.cuda.synchronize()
        ta = time.perf_counter()
        dev_in.copy_(hd, non_blocking=True)
        torch.cuda.synchronize()
        tb = time.perf_counter()
        hF.copy_(F, non_blocking=True)
        hI.copy_(I, non_blocking=True)
        torch.cuda.synchronize()
        tc = time.perf_counter()
        del dev_in
        e2e_parts = {"set_ic_ms": ic_ms, "collapse_host_out_ms": col_ms, "graph_ms": ms,
                     "d2h_ms_est": d2h_ms, "h2d_gbs_incl_phi0": d32.nbytes / (ic_ms / 1e3) / 1e9,
                     "d2h_gbs_est": 8 * n ** 3 / (d2h_ms / 1e3) / 1e9,
                     "torch_copy_same_buffers": {"h2d_gbs": d32.nbytes / (tb - ta) / 1e9,
                                                 "d2h_gbs": 8 * n ** 3 / (tc - tb) / 1e9}}
    barrier()
    if not args.no_e2e:
        e2e_s, _ = replica_value(e2e_s, updates, ws, "cuda")
    stats = plan.stats()
    kernels_per_call = pin.pin_kernels_per_call(plan.handle)
    pin_schedule = pin.pin_get_schedule(plan.handle)
    radix = plan.radix()

    # roofline of the dominant pass (algorithmic bytes per launch, one launch per radius)
    fused = kernels_per_call == 4 * S
    per_launch_ms = pass_ms / S
    alg = algorithmic_bytes(n, fused, bool(args.velocities))
    names = ["x", "y", "z", "roots"]
    if fused:
        names[3] = "redo"  # the z pass computes the collapse times; only the FP64 redo follows
    dom = int(np.argmax(per_launch_ms))
    peak, peak_kind = _peaks()
    achieved = alg[names[dom]] / (per_launch_ms[dom] / 1e3) / 1e9
    passes = {nm: {"ms_per_launch": float(per_launch_ms[i]),
                   "alg_bytes_per_launch": alg[nm],
                   "gbs": alg[nm] / (per_launch_ms[i] / 1e3) / 1e9 if alg[nm] else None,
                   "frac": alg[nm] / (per_launch_ms[i] / 1e3) / 1e9 / peak if alg[nm] else None}
              for i, nm in enumerate(names)}
    # the whole radius loop: every pass's algorithmic bytes over the step time
    step_bytes = S * sum(alg.values())
    whole_step = {"alg_bytes_per_update": step_bytes / updates,
                  "gbs": step_bytes / (ms / 1e3) / 1e9,
                  "frac": step_bytes / (ms / 1e3) / 1e9 / peak}
    if ws > 1:
        dist.barrier()
    plan.close()
    configs = None
    if rank == 0 and ws == 1 and not args.no_configs and not args.grid and not args.nscales:
        # the smaller workloads, device-timed, after the main plan is gone
        configs = {k: measure_config(c, max(3, args.steps), args.warmup, tune=not args.no_tune)
                   for k, c in CONFIGS.items()}
    if rank == 0:
        clocks = clk.summary()
        cb = cpu_baseline(S) if ws == 1 and not args.no_cpu else None
        line = {
            "metric": METRIC if n == WORKLOAD["n"] else METRIC.replace("768^3", "%d^3" % n),
            "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "best_ms_per_step": min(step_ms),
            "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": dict(_config(w), velocities=bool(args.velocities),
                           tiles={"x": tiles[0], "y": tiles[1], "radix_x": radix[0], "radix_y": radix[1],
                                  "radix_shapes": {"x": pin.pin_radix_shape(n, radix[0]),
                                                   "y": pin.pin_radix_shape(n, radix[1])},
                                  "tuned": not (args.no_tune or args.tiles or args.radix)},
                           schedule=pin_schedule),
            "roofline": dict(roofline(names[dom], per_launch_ms[dom], n, bool(args.velocities), fused,
                                      achieved, peak, peak_kind, clocks, passes), step=whole_step),
            "cpu_baseline": cb,
            "e2e": None if args.no_e2e else {"value": updates * ws / e2e_s, "unit": UNIT,
                    "h2d_bytes_per_step": int(d32.nbytes), "d2h_bytes_per_step": int(8 * n ** 3),
                    "ms_per_step": e2e_s * 1e3, "parts": e2e_parts},
            "gpu_launches": int(args.steps * kernels_per_call),
            "clocks": clocks,
            "fp64_redo": {"eig": stats["eig_fp64_redo"], "root": stats["root_fp64_redo"],
                          "particle_scales": int(stats["collapse_calls"]) * updates},
            "configs": configs,
        }
        print(json.dumps(line), flush=True)
    if ws > 1:
        dist.destroy_process_group()
    return 0


# 64 realisations of 128^3 (box 256 Mpc/h, seeds 100..163), 25 radii 40 -> 2 Mpc/h
ENSEMBLE = dict(n=128, box=256.0, seed0=100, count=64, nscales=25, r_min=2.0, r_max=40.0)


def run_ensemble(args):
    """Batched ensemble: all realisations in one plan (one launch per pass per
    radius) against the same realisations run one at a time through a plain
    plan; realisations/hour for both, same results bit for bit."""
    import torch
    from paper_1305_1505_gb300 import ic, pin
    e = ENSEMBLE
    n, B = e["n"], e["count"]
    radii = ic.log_radii(e["r_min"], e["r_max"], e["nscales"])
    fields = np.stack([ic.delta_k(n, e["box"], e["seed0"] + i, dtype=np.complex64) for i in range(B)])
    dk = torch.from_numpy(fields).cuda()
    stream = torch.cuda.Stream()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    bplan = pin.Plan(n, e["box"], radii, stream=stream, batch=B)
    if not args.no_tune:
        bplan.autotune(reps=5)
    Fb = torch.empty((B, n, n, n), dtype=torch.float32, device="cuda")
    Ib = torch.empty((B, n, n, n), dtype=torch.int32, device="cuda")
    torch.cuda.synchronize()

    def batched():
        pin.pin_set_ic(bplan.handle, dk.data_ptr(), pin.PIN_C64, 1)
        pin.pin_collapse_times(bplan.handle, Fb.data_ptr(), Ib.data_ptr(), 1)

    for _ in range(args.warmup):
        batched()
    bplan.sync()
    torch.cuda.synchronize()
    ev0.record(stream)
    for _ in range(args.steps):
        batched()
    ev1.record(stream)
    torch.cuda.synchronize()
    t_batch = ev0.elapsed_time(ev1) / 1e3 / args.steps

    splan = pin.Plan(n, e["box"], radii, stream=stream)
    if not args.no_tune:
        splan.autotune(reps=5)
    Fs = torch.empty((B, n, n, n), dtype=torch.float32, device="cuda")
    Is = torch.empty((B, n, n, n), dtype=torch.int32, device="cuda")

    def sequential():
        for i in range(B):
            pin.pin_set_ic(splan.handle, dk[i].data_ptr(), pin.PIN_C64, 1)
            pin.pin_collapse_times(splan.handle, Fs[i].data_ptr(), Is[i].data_ptr(), 1)

    for _ in range(args.warmup):
        sequential()
    splan.sync()
    torch.cuda.synchronize()
    ev0.record(stream)
    for _ in range(args.steps):
        sequential()
    ev1.record(stream)
    torch.cuda.synchronize()
    t_seq = ev0.elapsed_time(ev1) / 1e3 / args.steps
    same = bool(torch.equal(Fb, Fs) and torch.equal(Ib, Is))
    upd = B * n ** 3 * e["nscales"]
    line = {"metric": "realisations/hour, batched ensemble of 64 x 128^3 x 25 radii",
            "value": B / t_batch * 3600, "unit": "realisations/hour", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_batch * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": "64 realisations 128^3, box 256 Mpc/h, seeds 100..163, "
                                   "25 radii 40->2 Mpc/h", "batch": B},
            "sequential": {"value": B / t_seq * 3600, "unit": "realisations/hour",
                           "ms_per_step": t_seq * 1e3},
            "speedup_vs_sequential": t_seq / t_batch,
            "updates_per_s": {"batched": upd / t_batch, "sequential": upd / t_seq},
            "identical_results": same,
            "gpu_launches": int(args.steps * pin.pin_kernels_per_call(bplan.handle))}
    print(json.dumps(line), flush=True)
    bplan.close()
    splan.close()
    return 0


# bytes each particle costs the fragmentation front end: four radix passes
# (histogram key read 4 B each; scatter: pass 0 reads F 4 B and writes key +
# index 8 B, passes 1-2 read and write 8 B, pass 3 reads 8 B and writes the
# index 4 B) and the neighbour count (F read 4 B, count write 1 B)
FRAGMENT_BYTES = 4 * 4 + (4 + 8) + 2 * (8 + 8) + (8 + 4) + (4 + 1)


def run_fragment(args):
    """Fragmentation front end (Sec. 2.1.2) on the 768^3 x 40 workload: one
    pin_collapse_times (untimed), then pin_fragment_order timed on the device
    (order and neighbour counts, device outputs), end to end with host
    outputs, and the oracle on a 128^3 block of the same F_max field."""
    import torch
    from paper_1305_1505_gb300 import ic, pin
    w = dict(WORKLOAD)
    if args.grid:
        w["n"], w["box"] = args.grid, 4.0 * args.grid
    n = w["n"]
    radii = ic.log_radii(w["r_min"], w["r_max"], w["nscales"])
    stream = torch.cuda.Stream()
    plan = pin.Plan(n, w["box"], radii, stream=stream)
    plan.set_ic(torch.from_numpy(ic.delta_k(n, w["box"], w["seed"], dtype=np.complex64)).cuda())
    F, _ = plan.collapse_times()
    order = torch.empty(n ** 3, dtype=torch.int32, device="cuda")
    nb = torch.empty((n, n, n), dtype=torch.uint8, device="cuda")
    torch.cuda.synchronize()

    def step():
        pin.pin_fragment_order(plan.handle, order.data_ptr(), nb.data_ptr(), 1)

    for _ in range(args.warmup):
        step()
    plan.sync()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    with ClockSampler(torch.cuda.current_device()) as clk:
        ev0.record(stream)
        for _ in range(args.steps):
            step()
        ev1.record(stream)
        torch.cuda.synchronize()
    t = ev0.elapsed_time(ev1) / 1e3 / args.steps
    e2e = None
    if not args.no_e2e:
        ho = torch.empty(n ** 3, dtype=torch.int32).pin_memory()
        hn = torch.empty((n, n, n), dtype=torch.uint8).pin_memory()
        pin.pin_fragment_order(plan.handle, ho.data_ptr(), hn.data_ptr(), 0)
        reps = max(1, min(args.steps, 3))
        t0 = time.perf_counter()
        for _ in range(reps):
            pin.pin_fragment_order(plan.handle, ho.data_ptr(), hn.data_ptr(), 0)
        te = (time.perf_counter() - t0) / reps
        e2e = {"value": n ** 3 / te, "unit": "particles/s", "h2d_bytes_per_step": 0,
               "d2h_bytes_per_step": int(5 * n ** 3)}
    cb = None
    if not args.no_cpu:
        import oracle
        m = min(128, n)
        block = F[:m, :m, :m].contiguous().cpu().numpy()
        t0 = time.perf_counter()
        oracle.fragment_order(block)
        tc = time.perf_counter() - t0
        cb = {"value": m ** 3 / tc, "unit": "particles/s", "cores": 1, "kind": "oracle",
              "sample": "%d^3 block of the same F_max field (numpy lexsort + rolls), %.1f s" % (m, tc)}
    peak, peak_kind = _peaks()
    achieved = FRAGMENT_BYTES * n ** 3 / t / 1e9
    line = {"metric": "fragmentation order (particles/s) at %d^3" % n, "value": n ** 3 / t,
            "unit": "particles/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": t * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "u32", "data": "synthetic",
            "config": {"workload": "F_max of the %d^3 x %d collapse workload, seed %d" % (n, w["nscales"], w["seed"]),
                       "l2": "inputs larger than L2 (F_max %.1f GB, sort buffers %.1f GB)"
                             % (4 * n ** 3 / 1e9, 16 * n ** 3 / 1e9)},
            "roofline": {"bound": "hbm", "kernel": "fragment_order (4 radix passes + neighbour count)",
                         "achieved": achieved, "peak": peak, "peak_kind": peak_kind, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": None,
                         "alg_bytes_per_particle": FRAGMENT_BYTES},
            "cpu_baseline": cb, "e2e": e2e,
            "gpu_launches": int(args.steps * 21), "clocks": clk.summary()}
    print(json.dumps(line), flush=True)
    plan.close()
    return 0


# bytes per particle of one pin_displacements_2lpt call (H ~ N^3/2 complex =
# 4 B per particle per spectrum): the unsmoothed Hessian passes (x 4 spectra,
# y 9, z reads 6 and writes the 4-byte source S), the forward transform of S
# (z reads S and writes a spectrum, y and x read and write one each), Phi2
# (read and write one), and the gradient passes (x 3 spectra, y 5, z reads 3
# and writes 12 bytes)
LPT2_BYTES = 16 + 36 + 28 + 8 + 8 + 8 + 8 + 12 + 20 + 24


def run_2lpt(args):
    """Second-order LPT displacement of the unsmoothed 768^3 field, timed on
    the device (output in device memory) and end to end (host output)."""
    import torch
    from paper_1305_1505_gb300 import ic, pin
    w = dict(WORKLOAD)
    if args.grid:
        w["n"], w["box"] = args.grid, 4.0 * args.grid
    n = w["n"]
    stream = torch.cuda.Stream()
    plan = pin.Plan(n, w["box"], [w["r_max"]], stream=stream)
    d32 = ic.delta_k(n, w["box"], w["seed"], dtype=np.complex64)
    plan.set_ic(torch.from_numpy(d32).cuda())
    if not args.no_tune:
        plan.autotune(reps=5)
    out = torch.empty((3, n, n, n), dtype=torch.float32, device="cuda")
    torch.cuda.synchronize()

    def step():
        pin.pin_displacements_2lpt(plan.handle, out.data_ptr(), 1)

    for _ in range(args.warmup):
        step()
    plan.sync()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    with ClockSampler(torch.cuda.current_device()) as clk:
        ev0.record(stream)
        for _ in range(args.steps):
            step()
        ev1.record(stream)
        torch.cuda.synchronize()
    t = ev0.elapsed_time(ev1) / 1e3 / args.steps
    e2e = None
    if not args.no_e2e:
        hd = torch.from_numpy(d32).pin_memory()
        ho = torch.empty((3, n, n, n), dtype=torch.float32).pin_memory()
        reps = max(1, min(args.steps, 3))
        t0 = time.perf_counter()
        for _ in range(reps):
            pin.pin_set_ic(plan.handle, hd.data_ptr(), pin.PIN_C64, 0)
            pin.pin_displacements_2lpt(plan.handle, ho.data_ptr(), 0)
        te = (time.perf_counter() - t0) / reps
        e2e = {"value": n ** 3 / te, "unit": "particles/s", "h2d_bytes_per_step": int(d32.nbytes),
               "d2h_bytes_per_step": int(12 * n ** 3)}
    cb = None
    if not args.no_cpu:
        import oracle
        m = min(128, n)
        dm = ic.delta_k(m, 4.0 * m, w["seed"])
        t0 = time.perf_counter()
        oracle.displacement_2lpt(dm, 4.0 * m)
        tc = time.perf_counter() - t0
        cb = {"value": m ** 3 / tc, "unit": "particles/s", "cores": os.cpu_count(), "kind": "oracle",
              "sample": "%d^3 grid with the same 4 Mpc/h cells, FP64, %.1f s" % (m, tc)}
    peak, peak_kind = _peaks()
    achieved = LPT2_BYTES * n ** 3 / t / 1e9
    line = {"metric": "2LPT displacement (particles/s) at %d^3" % n, "value": n ** 3 / t,
            "unit": "particles/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": t * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": "%d^3 grid, box %g Mpc/h, seed %d, unsmoothed" % (n, w["box"], w["seed"]),
                       "l2": "inputs larger than L2 (spectra %.1f GB each)" % (8 * n * n * (n // 2 + 1) / 1e9)},
            "roofline": {"bound": "hbm", "kernel": "2LPT passes (11 kernels)", "achieved": achieved,
                         "peak": peak, "peak_kind": peak_kind, "unit": "GB/s", "frac": achieved / peak,
                         "traffic": None, "alg_bytes_per_particle": LPT2_BYTES},
            "cpu_baseline": cb, "e2e": e2e, "gpu_launches": int(args.steps * 11), "clocks": clk.summary()}
    print(json.dumps(line), flush=True)
    plan.close()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU-baseline leg")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer end-to-end leg")
    ap.add_argument("--no-tune", action="store_true",
                    help="run the default x/y tile widths instead of the tuned ones")
    ap.add_argument("--grid", type=int, default=0,
                    help="grid side for profiling captures (box = 4 Mpc/h per cell); default 768")
    ap.add_argument("--nscales", type=int, default=0, help="number of radii; default 40")
    ap.add_argument("--velocities", action="store_true",
                    help="also keep v_max (the displacement smoothed on R_max): 9 fields per radius")
    ap.add_argument("--workload", default="paper",
                    choices=["paper", "config1", "config2", "ensemble", "serve", "fragment", "2lpt"],
                    help="paper: 768^3 x 40 (the metric); config1: 64^3 x 20; config2: 256^3 x 30; "
                         "ensemble: 64 x 128^3 batched vs sequential; "
                         "serve: 600 Poisson requests of mixed sizes, p50/p99 (--requests, --rate); "
                         "fragment: the fragmentation front end on the 768^3 F_max field; "
                         "2lpt: the second-order displacement of the 768^3 field")
    ap.add_argument("--schedule", type=int, default=0,
                    help="radius schedule (pin_set_schedule): 0 serial, 1 z(s) beside x(s+1), "
                         "2 z(s) beside x and y of s+1")
    ap.add_argument("--tiles", default="", help="force the x,y tile widths (e.g. 8,8) instead of tuning")
    ap.add_argument("--radix", default="", help="force the x,y radix schedules (e.g. 1,1) instead of tuning")
    ap.add_argument("--requests", type=int, default=600, help="serve: number of requests")
    ap.add_argument("--rate", type=float, default=2.0, help="serve: mean arrivals per second")
    ap.add_argument("--no-configs", action="store_true",
                    help="default workload: skip the smaller workloads measured after it")
    args = ap.parse_args()
    if args.workload == "ensemble":
        return run_ensemble(args)
    if args.workload == "fragment":
        return run_fragment(args)
    if args.workload == "2lpt":
        return run_2lpt(args)
    if args.workload in CONFIGS:
        return run_config(args, args.workload)
    if args.workload == "serve":
        from paper_1305_1505_gb300 import serve
        line = serve.measure_serving(args.requests, args.rate)
        nom = line["nominal"]
        line.update({"value": nom["served"]["p99_s"], "unit": "s (p99 latency)", "higher_is_better": False,
                     "n_gpus": 1, "dtype": "f32", "data": "synthetic", "vs_baseline": None})
        print(json.dumps(line), flush=True)
        return 0
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
