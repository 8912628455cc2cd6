"""Thin ctypes binding of libpin.so (C-ABI in include/pin.h).

Argument marshalling only: every step of the collapse-time path runs in the
CUDA kernels of csrc/.  There is no CPU fallback; if the native library is
missing or no GPU is present the calls raise.

The functions keep the C names (pin_plan, pin_set_ic, pin_collapse_times,
pin_hessian, pin_displacements, pin_sync, ...).  `Plan` and `collapse_times`
are conveniences over them that take PyTorch device tensors (PyTorch provides
device memory and streams only).
"""
import ctypes
import os

import numpy as np

from . import build as _build

PIN_OK, PIN_EINVAL, PIN_ENOMEM, PIN_ECUDA, PIN_EBUSY, PIN_ETIMEOUT, PIN_ESTATE = range(7)
PIN_CORR_NONE, PIN_CORR_SPHERE = 0, 1
PIN_FP32_FALLBACK64, PIN_FP64 = 0, 1
PIN_C64, PIN_C128 = 0, 1
PIN_TUNE_FORCE = 1

MAX_SCALES = 64


class PinError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s (status %d): %s" % (_strerror(status), status, msg))
        self.status = status


class pin_plan_desc(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("box", ctypes.c_double), ("nscales", ctypes.c_int),
                ("radii", ctypes.POINTER(ctypes.c_double)), ("correction", ctypes.c_int),
                ("precision", ctypes.c_int), ("stream", ctypes.c_void_p),
                ("batch", ctypes.c_int), ("velocities", ctypes.c_int)]


class pin_spectrum(ctypes.Structure):
    _fields_ = [("ns", ctypes.c_double), ("gamma", ctypes.c_double), ("sigma8", ctypes.c_double)]


def spectrum(ns=0.96, gamma=0.21, sigma8=0.8):
    return pin_spectrum(ns, gamma, sigma8)


class pin_stats(ctypes.Structure):
    _fields_ = [("eig_fp64_redo", ctypes.c_uint64), ("root_fp64_redo", ctypes.c_uint64),
                ("fp64_queue_overflow", ctypes.c_uint64), ("collapse_calls", ctypes.c_uint64)]


# every symbol include/pin.h declares
EXPORTS = ("pin_plan", "pin_footprint_bytes", "pin_set_ic", "pin_collapse_times", "pin_collapse_times_f64",
           "pin_hessian",
           "pin_displacements", "pin_sync", "pin_get_stats", "pin_kernels_per_call",
           "pin_profile", "pin_pass_times", "pin_collapse_times_noalloc", "pin_velocities",
           "pin_fragment_order", "pin_displacements_2lpt", "pin_set_ic_seed", "pin_tile_options",
           "pin_tile_options_radix", "pin_radix_schedules", "pin_radix_shape", "pin_get_radix", "pin_set_radix",
           "pin_get_tiles", "pin_set_tiles", "pin_autotune", "pin_noalloc_status", "pin_set_radii", "pin_set_schedule",
           "pin_get_schedule", "pin_set_wait_budget",
           "pin_debug_fail_alloc", "pin_strerror", "pin_last_error", "pin_destroy")

_lib = None


def load(path=None):
    """Loads libpin.so (building it in-tree if stale) and declares signatures."""
    global _lib
    if _lib is not None:
        return _lib
    # PIN_LIBRARY selects another build of the same sources (e.g. a tuning variant)
    path = path or os.environ.get("PIN_LIBRARY") or _build.ensure_pin()
    if not os.path.exists(path):
        raise RuntimeError("libpin.so not found at %s; run __graft_entry__.build()" % path)
    L = ctypes.CDLL(path)
    P = ctypes.c_void_p
    L.pin_plan.argtypes = [ctypes.POINTER(P), ctypes.POINTER(pin_plan_desc)]
    L.pin_plan.restype = ctypes.c_int
    L.pin_footprint_bytes.argtypes = [ctypes.POINTER(pin_plan_desc)]
    L.pin_footprint_bytes.restype = ctypes.c_size_t
    L.pin_set_ic.argtypes = [P, P, ctypes.c_int, ctypes.c_int]
    L.pin_set_ic.restype = ctypes.c_int
    L.pin_collapse_times.argtypes = [P, P, P, ctypes.c_int]
    L.pin_collapse_times.restype = ctypes.c_int
    L.pin_collapse_times_f64.argtypes = [P, P, P, ctypes.c_int]
    L.pin_collapse_times_f64.restype = ctypes.c_int
    L.pin_velocities.argtypes = [P, P, ctypes.c_int]
    L.pin_velocities.restype = ctypes.c_int
    L.pin_fragment_order.argtypes = [P, P, P, ctypes.c_int]
    L.pin_fragment_order.restype = ctypes.c_int
    L.pin_displacements_2lpt.argtypes = [P, P, ctypes.c_int]
    L.pin_displacements_2lpt.restype = ctypes.c_int
    L.pin_set_ic_seed.argtypes = [P, ctypes.c_uint64, ctypes.POINTER(pin_spectrum)]
    L.pin_set_ic_seed.restype = ctypes.c_int
    L.pin_hessian.argtypes = [P, ctypes.c_int, P, ctypes.c_int]
    L.pin_hessian.restype = ctypes.c_int
    L.pin_displacements.argtypes = [P, P, ctypes.c_int]
    L.pin_displacements.restype = ctypes.c_int
    L.pin_sync.argtypes = [P, ctypes.c_int64]
    L.pin_sync.restype = ctypes.c_int
    L.pin_get_stats.argtypes = [P, ctypes.POINTER(pin_stats)]
    L.pin_get_stats.restype = ctypes.c_int
    L.pin_kernels_per_call.argtypes = [P]
    L.pin_kernels_per_call.restype = ctypes.c_int
    L.pin_profile.argtypes = [P, ctypes.c_int]
    L.pin_profile.restype = ctypes.c_int
    L.pin_pass_times.argtypes = [P, ctypes.POINTER(ctypes.c_double)]
    L.pin_pass_times.restype = ctypes.c_int
    IP = ctypes.POINTER(ctypes.c_int)
    L.pin_tile_options.argtypes = [ctypes.c_int, IP, IP]
    L.pin_tile_options.restype = ctypes.c_int
    L.pin_tile_options_radix.argtypes = [ctypes.c_int, ctypes.c_int, IP, IP]
    L.pin_tile_options_radix.restype = ctypes.c_int
    L.pin_radix_schedules.argtypes = []
    L.pin_radix_schedules.restype = ctypes.c_int
    L.pin_radix_shape.argtypes = [ctypes.c_int, ctypes.c_int, IP, IP, IP]
    L.pin_radix_shape.restype = ctypes.c_int
    L.pin_get_radix.argtypes = [P, IP, IP]
    L.pin_get_radix.restype = ctypes.c_int
    L.pin_set_radix.argtypes = [P, ctypes.c_int, ctypes.c_int]
    L.pin_set_radix.restype = ctypes.c_int
    L.pin_get_tiles.argtypes = [P, IP, IP]
    L.pin_get_tiles.restype = ctypes.c_int
    L.pin_set_tiles.argtypes = [P, ctypes.c_int, ctypes.c_int]
    L.pin_set_tiles.restype = ctypes.c_int
    L.pin_autotune.argtypes = [P, ctypes.c_int, ctypes.c_int, IP, IP]
    L.pin_autotune.restype = ctypes.c_int
    L.pin_collapse_times_noalloc.argtypes = [P, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                             ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                                             ctypes.c_int, P, P, P]
    L.pin_collapse_times_noalloc.restype = ctypes.c_int
    L.pin_noalloc_status.argtypes = [IP, ctypes.POINTER(ctypes.c_uint64)]
    L.pin_noalloc_status.restype = ctypes.c_int
    L.pin_set_radii.argtypes = [P, ctypes.c_int, ctypes.POINTER(ctypes.c_double)]
    L.pin_set_radii.restype = ctypes.c_int
    L.pin_set_schedule.argtypes = [P, ctypes.c_int]
    L.pin_set_schedule.restype = ctypes.c_int
    L.pin_get_schedule.argtypes = [P]
    L.pin_get_schedule.restype = ctypes.c_int
    L.pin_set_wait_budget.argtypes = [P, ctypes.c_int64]
    L.pin_set_wait_budget.restype = ctypes.c_int
    L.pin_debug_fail_alloc.argtypes = [ctypes.c_int]
    L.pin_debug_fail_alloc.restype = None
    L.pin_strerror.argtypes = [ctypes.c_int]
    L.pin_strerror.restype = ctypes.c_char_p
    L.pin_last_error.argtypes = [P]
    L.pin_last_error.restype = ctypes.c_char_p
    L.pin_destroy.argtypes = [P]
    L.pin_destroy.restype = None
    _lib = L
    return L


def _strerror(status):
    try:
        return load().pin_strerror(status).decode()
    except Exception:  # library unavailable while formatting an error
        return "status"


def _check(status, plan=None):
    if status != PIN_OK:
        msg = ""
        if plan is not None:
            msg = load().pin_last_error(plan).decode(errors="replace")
        raise PinError(status, msg)


def grid_shape(n):
    """(nx, ny, nz) from a side length or a 3-tuple."""
    if np.ndim(n) == 0:
        return (int(n),) * 3
    nx, ny, nz = (int(v) for v in n)
    return nx, ny, nz


def make_desc(n, box, radii, correction=PIN_CORR_SPHERE, stream=None, batch=1, velocities=False,
              precision=PIN_FP32_FALLBACK64):
    """n: the grid side, or (nx, ny, nz) for a non-cubic grid (cubic cells:
    box is the side along x)."""
    r = np.ascontiguousarray(radii, dtype=np.float64)
    nx, ny, nz = grid_shape(n)
    d = pin_plan_desc(nx, ny, nz, float(box), int(r.size),
                      r.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), int(correction),
                      int(precision), ctypes.c_void_p(stream) if stream else None, int(batch),
                      1 if velocities else 0)
    d._radii_keepalive = r
    return d


# ---- C names ---------------------------------------------------------------

def pin_plan(desc):
    h = ctypes.c_void_p()
    st = load().pin_plan(ctypes.byref(h), ctypes.byref(desc))
    _check(st)
    return h


def pin_footprint_bytes(desc):
    return load().pin_footprint_bytes(ctypes.byref(desc))


def pin_set_ic(plan, delta_k_ptr, dtype, on_device):
    _check(load().pin_set_ic(plan, ctypes.c_void_p(delta_k_ptr), dtype, int(on_device)), plan)


def pin_collapse_times(plan, fmax_ptr, idx_ptr, on_device):
    _check(load().pin_collapse_times(plan, ctypes.c_void_p(fmax_ptr), ctypes.c_void_p(idx_ptr),
                                     int(on_device)), plan)


def pin_collapse_times_f64(plan, fmax_ptr, idx_ptr, on_device):
    _check(load().pin_collapse_times_f64(plan, ctypes.c_void_p(fmax_ptr), ctypes.c_void_p(idx_ptr),
                                         int(on_device)), plan)


def pin_velocities(plan, out_ptr, on_device):
    _check(load().pin_velocities(plan, ctypes.c_void_p(out_ptr), int(on_device)), plan)


def pin_fragment_order(plan, order_ptr, n_before_ptr, on_device):
    _check(load().pin_fragment_order(plan, ctypes.c_void_p(order_ptr) if order_ptr else None,
                                     ctypes.c_void_p(n_before_ptr) if n_before_ptr else None,
                                     int(on_device)), plan)


def pin_set_ic_seed(plan, seed, spec=None):
    sp = spec if spec is not None else spectrum()
    _check(load().pin_set_ic_seed(plan, ctypes.c_uint64(int(seed)), ctypes.byref(sp)), plan)


def pin_displacements_2lpt(plan, out_ptr, on_device):
    _check(load().pin_displacements_2lpt(plan, ctypes.c_void_p(out_ptr), int(on_device)), plan)


def pin_hessian(plan, scale, out_ptr, on_device):
    _check(load().pin_hessian(plan, int(scale), ctypes.c_void_p(out_ptr), int(on_device)), plan)


def pin_displacements(plan, out_ptr, on_device):
    _check(load().pin_displacements(plan, ctypes.c_void_p(out_ptr), int(on_device)), plan)


def pin_sync(plan, timeout_ns=-1):
    return load().pin_sync(plan, int(timeout_ns))


def pin_get_stats(plan):
    s = pin_stats()
    _check(load().pin_get_stats(plan, ctypes.byref(s)), plan)
    return dict(eig_fp64_redo=s.eig_fp64_redo, root_fp64_redo=s.root_fp64_redo,
                fp64_queue_overflow=s.fp64_queue_overflow, collapse_calls=s.collapse_calls)


def pin_kernels_per_call(plan):
    return load().pin_kernels_per_call(plan)


def pin_profile(plan, enable):
    _check(load().pin_profile(plan, int(enable)), plan)


def pin_pass_times(plan):
    """[x, y, z, roots] device milliseconds of the last call, summed over radii."""
    ms = (ctypes.c_double * 4)()
    _check(load().pin_pass_times(plan, ms), plan)
    return list(ms)


def pin_tile_options(n):
    """Tile widths (columns per block) the x/y pass over lines of n points can
    run, the default first."""
    opts = (ctypes.c_int * 2)()
    k = ctypes.c_int(0)
    _check(load().pin_tile_options(int(n), opts, ctypes.byref(k)))
    return list(opts[:k.value])


def pin_tile_options_radix(n, radix):
    opts = (ctypes.c_int * 2)()
    k = ctypes.c_int(0)
    _check(load().pin_tile_options_radix(int(n), int(radix), opts, ctypes.byref(k)))
    return list(opts[:k.value])


def pin_radix_schedules():
    return load().pin_radix_schedules()


def pin_radix_shape(n, radix):
    """(E, P1, P2) of radix schedule `radix` for lines of n points."""
    e, p1, p2 = ctypes.c_int(0), ctypes.c_int(0), ctypes.c_int(0)
    _check(load().pin_radix_shape(int(n), int(radix), ctypes.byref(e), ctypes.byref(p1), ctypes.byref(p2)))
    return e.value, p1.value, p2.value


def pin_get_radix(plan):
    x, y = ctypes.c_int(0), ctypes.c_int(0)
    _check(load().pin_get_radix(plan, ctypes.byref(x), ctypes.byref(y)), plan)
    return x.value, y.value


def pin_set_radix(plan, vx, vy):
    _check(load().pin_set_radix(plan, int(vx), int(vy)), plan)


def pin_get_tiles(plan):
    """(x-pass, y-pass) tile widths the plan runs."""
    x, y = ctypes.c_int(0), ctypes.c_int(0)
    _check(load().pin_get_tiles(plan, ctypes.byref(x), ctypes.byref(y)), plan)
    return x.value, y.value


def pin_set_tiles(plan, tc_x, tc_y):
    _check(load().pin_set_tiles(plan, int(tc_x), int(tc_y)), plan)


def pin_autotune(plan, reps=3, flags=0):
    """Times the candidate tile widths of the x and y passes and keeps the
    fastest (kept per grid shape for the process); returns (tc_x, tc_y)."""
    x, y = ctypes.c_int(0), ctypes.c_int(0)
    _check(load().pin_autotune(plan, int(reps), int(flags), ctypes.byref(x), ctypes.byref(y)), plan)
    return x.value, y.value


def pin_collapse_times_noalloc(delta_k_ptr, dtype, n, box, radii, correction, fmax_ptr, idx_ptr,
                               stream_ptr=None):
    """No-allocation collapse times for n <= 64 (device pointers in and out);
    for callers that cannot allocate device memory at call time."""
    r = np.ascontiguousarray(radii, dtype=np.float64)
    st = load().pin_collapse_times_noalloc(ctypes.c_void_p(delta_k_ptr), int(dtype), int(n),
                                           float(box), int(r.size),
                                           r.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                           int(correction), ctypes.c_void_p(fmax_ptr),
                                           ctypes.c_void_p(idx_ptr), ctypes.c_void_p(stream_ptr))
    _check(st)


def pin_noalloc_status():
    """(status, wait_failed, [eig redo, root redo, queue overflow]) recorded by
    the last pin_collapse_times_noalloc on the current device; call after its
    stream has completed.  status is PIN_ECUDA when a bounded transfer wait
    gave up (its outputs are then invalid)."""
    w = ctypes.c_int(0)
    c = (ctypes.c_uint64 * 3)()
    st = load().pin_noalloc_status(ctypes.byref(w), c)
    if st not in (PIN_OK, PIN_ECUDA):
        _check(st)
    return st, w.value, list(c)


def pin_set_radii(plan, radii):
    r = np.ascontiguousarray(radii, dtype=np.float64)
    _check(load().pin_set_radii(plan, int(r.size), r.ctypes.data_as(ctypes.POINTER(ctypes.c_double))), plan)


def pin_set_schedule(plan, schedule):
    """Radius schedule: 0 serial, 1 z(s) beside x(s+1), 2 z(s) beside x and
    y of s+1 (second V buffer)."""
    _check(load().pin_set_schedule(plan, int(schedule)), plan)


def pin_get_schedule(plan):
    return load().pin_get_schedule(plan)


def pin_set_wait_budget(plan, cycles):
    """Budget (SM clocks) of the x/y passes' bounded transfer waits; 0 restores
    the default (2^31 clocks)."""
    _check(load().pin_set_wait_budget(plan, int(cycles)), plan)


def pin_debug_fail_alloc(nth):
    """Makes the nth later device allocation of pin_plan fail (nth < 0: off)."""
    load().pin_debug_fail_alloc(int(nth))


def pin_strerror(status):
    return load().pin_strerror(status).decode()


def pin_last_error(plan):
    return load().pin_last_error(plan).decode(errors="replace")


def pin_destroy(plan):
    load().pin_destroy(plan)


# ---- conveniences over PyTorch device memory --------------------------------

class Plan:
    """Owns one pin plan; methods take torch tensors (device or host)."""

    def __init__(self, n, box, radii, correction=PIN_CORR_SPHERE, stream=None, batch=1,
                 velocities=False, precision=PIN_FP32_FALLBACK64):
        """n: grid side, or (nx, ny, nz) for a non-cubic grid with cubic cells
        (box is the side along x)."""
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("pin needs a CUDA device; none is available")
        self.shape = grid_shape(n)
        self.n = self.shape[0]
        self.box = float(box)
        self.batch = int(batch)
        self.radii = np.ascontiguousarray(radii, dtype=np.float64)
        s = stream.cuda_stream if stream is not None else None
        self._desc = make_desc(self.shape, self.box, self.radii, correction, s, self.batch, velocities,
                               precision)
        self.handle = pin_plan(self._desc)

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and h.value:
            try:
                pin_destroy(h)
            except Exception:
                pass
            self.handle = None

    def close(self):
        self.__del__()

    def set_ic(self, delta_k):
        """delta_k: (n, n, n//2+1) complex64/complex128 tensor or numpy array, or
        (batch, n, n, n//2+1) for a batched plan."""
        import torch
        if isinstance(delta_k, np.ndarray):
            a = np.ascontiguousarray(delta_k)
            dt = PIN_C64 if a.dtype == np.complex64 else PIN_C128
            if a.dtype not in (np.complex64, np.complex128):
                raise TypeError("delta_k must be complex64 or complex128")
            pin_set_ic(self.handle, a.ctypes.data, dt, 0)
            return
        t = delta_k.contiguous()
        dt = {torch.complex64: PIN_C64, torch.complex128: PIN_C128}[t.dtype]
        if t.is_cuda:
            torch.cuda.current_stream().synchronize()  # producer stream -> plan stream
        pin_set_ic(self.handle, t.data_ptr(), dt, 1 if t.is_cuda else 0)
        if t.is_cuda:
            self.sync()

    def set_radii(self, radii):
        """Replaces the radius list (the plan's workspace is kept)."""
        r = np.ascontiguousarray(radii, dtype=np.float64)
        pin_set_radii(self.handle, r)
        self.radii = r

    def set_ic_seed(self, seed, ns=0.96, gamma=0.21, sigma8=0.8):
        """delta(k) generated on the device from `seed` (realisation b of a
        batch: seed + b), the seeded field of the input module."""
        pin_set_ic_seed(self.handle, seed, spectrum(ns, gamma, sigma8))

    def collapse_times(self, fmax=None, idx=None, sync=True):
        """Returns (F_max float32, scale_idx int32) tensors of shape (n,n,n),
        on the device unless host tensors are passed in.  With sync=False the
        work is only enqueued on the plan's stream (call .sync() before use)."""
        import torch
        shape = self.shape if self.batch == 1 else (self.batch,) + self.shape
        if fmax is None:
            fmax = torch.empty(shape, dtype=torch.float32, device="cuda")
        if idx is None:
            idx = torch.empty(shape, dtype=torch.int32, device=fmax.device)
        if fmax.is_cuda != idx.is_cuda:
            raise ValueError("F_max and scale_idx must both be on the device or both on the host")
        if fmax.is_cuda:
            torch.cuda.current_stream().synchronize()  # outputs allocated on torch's stream
        pin_collapse_times(self.handle, fmax.data_ptr(), idx.data_ptr(), 1 if fmax.is_cuda else 0)
        if sync and fmax.is_cuda:
            self.sync()
        return fmax, idx

    def collapse_times_f64(self):
        """(F_max float64, scale_idx int32) of a PIN_FP64 plan, on the device."""
        import torch
        F = torch.empty(self.shape, dtype=torch.float64, device="cuda")
        I = torch.empty(self.shape, dtype=torch.int32, device="cuda")
        torch.cuda.current_stream().synchronize()
        pin_collapse_times_f64(self.handle, F.data_ptr(), I.data_ptr(), 1)
        self.sync()
        return F, I

    def velocities(self):
        """(3, [batch,] n, n, n) displacement at R_max of the last collapse_times."""
        import torch
        shape = (3,) + self.shape if self.batch == 1 else (3, self.batch) + self.shape
        out = torch.empty(shape, dtype=torch.float32, device="cuda")
        torch.cuda.current_stream().synchronize()
        pin_velocities(self.handle, out.data_ptr(), 1)
        self.sync()
        return out

    def fragment_order(self, order=True, n_before=True):
        """(order, n_before) of the last collapse_times (Sec. 2.1.2): the
        particle indices in descending F_max (ties by index) as an (n^3,)
        int32 tensor, and per particle the number of its six neighbours that
        precede it, (n, n, n) uint8; either may be skipped (None)."""
        import torch
        o = torch.empty((int(np.prod(self.shape)),), dtype=torch.int32, device="cuda") if order else None
        c = torch.empty(self.shape, dtype=torch.uint8, device="cuda") if n_before else None
        torch.cuda.current_stream().synchronize()
        pin_fragment_order(self.handle, o.data_ptr() if o is not None else 0,
                           c.data_ptr() if c is not None else 0, 1)
        self.sync()
        return o, c

    def displacements_2lpt(self):
        """(3, n, n, n) second-order LPT displacement of the unsmoothed field."""
        import torch
        out = torch.empty((3,) + self.shape, dtype=torch.float32, device="cuda")
        torch.cuda.current_stream().synchronize()
        pin_displacements_2lpt(self.handle, out.data_ptr(), 1)
        self.sync()
        return out

    def hessian(self, scale):
        import torch
        out = torch.empty((6,) + self.shape, dtype=torch.float32, device="cuda")
        torch.cuda.current_stream().synchronize()
        pin_hessian(self.handle, scale, out.data_ptr(), 1)
        self.sync()
        return out

    def displacements(self):
        import torch
        out = torch.empty((3,) + self.shape, dtype=torch.float32, device="cuda")
        torch.cuda.current_stream().synchronize()
        pin_displacements(self.handle, out.data_ptr(), 1)
        self.sync()
        return out

    def sync(self, timeout_s=None):
        st = pin_sync(self.handle, -1 if timeout_s is None else int(timeout_s * 1e9))
        _check(st, self.handle)

    def tiles(self):
        """(x-pass, y-pass) tile widths in use."""
        return pin_get_tiles(self.handle)

    def radix(self):
        """(x-pass, y-pass) radix schedules in use."""
        return pin_get_radix(self.handle)

    def set_radix(self, vx=0, vy=0):
        pin_set_radix(self.handle, vx, vy)

    def set_tiles(self, tc_x=0, tc_y=0):
        """Forces tile widths (0: the default); each must be one of
        pin_tile_options of the pass's line length."""
        pin_set_tiles(self.handle, tc_x, tc_y)

    def autotune(self, reps=3, force=False):
        """Times the candidate tile widths on this plan and keeps the fastest;
        returns (tc_x, tc_y)."""
        return pin_autotune(self.handle, reps, PIN_TUNE_FORCE if force else 0)

    def stats(self):
        return pin_get_stats(self.handle)


def collapse_times(delta_k, radii, box, correction=PIN_CORR_SPHERE):
    """One-shot: (F_max, scale_idx) for the half-spectrum delta_k of shape
    (nx, ny, nz//2+1) (every supported nz is even; cubic cells, box along x)."""
    nx, ny, nh = delta_k.shape
    plan = Plan((nx, ny, 2 * (nh - 1)), box, radii, correction)
    try:
        plan.set_ic(delta_k)
        f, i = plan.collapse_times()
        plan.sync()
        return f, i
    finally:
        plan.close()
