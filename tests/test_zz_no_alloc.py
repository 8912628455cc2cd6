"""The no-allocation entry point (pin_collapse_times_noalloc) against
pin_collapse_times, through the C-ABI, on several calls in a row.

The entry point exists for callers that cannot allocate device memory at
call time: a serving pool that already owns the device's memory, code inside
an allocator hook, latency-critical code that cannot take cudaFree's
device-wide synchronisation.  Its workspace is one static device array shared
by all calls, so consecutive calls (a second input at the same size, then
smaller grids, C128 input and the uncorrected mode) also show that nothing of
an earlier call's contents leaks into a later one.  Both entry points build
the same tables and run the same kernels, so the results must agree bit for
bit; after each call the status getter must report no failed wait and no
overflow of the FP64 redo queue.  This file sorts last so that a run stopping
at its first failure has run everything else already."""
import numpy as np
import pytest

from paper_1305_1505_gb300 import ic, pin
from tests import parity

pytestmark = pytest.mark.gpu

# (n, box, seed, nscales, r_max, input dtype, correction), run in this order
CALLS = [
    (64, 100.0, 1, 20, 15.0, "c64", pin.PIN_CORR_SPHERE),
    (64, 100.0, 2, 20, 15.0, "c64", pin.PIN_CORR_SPHERE),
    (48, 96.0, 3, 12, 24.0, "c128", pin.PIN_CORR_SPHERE),
    (16, 64.0, 4, 8, 16.0, "c64", pin.PIN_CORR_NONE),
    (32, 64.0, 5, 10, 16.0, "c64", pin.PIN_CORR_SPHERE),
]


def _plan_path(d, n, box, radii, correction):
    import torch
    plan = pin.Plan(n, box, radii, correction)
    plan.set_ic(torch.from_numpy(d).cuda())
    F, I = plan.collapse_times()
    out = F.cpu().numpy().ravel(), I.cpu().numpy().ravel()
    plan.close()
    return out


def test_noalloc_equals_plan_path_on_consecutive_calls():
    import torch
    stream = torch.cuda.Stream()
    for n, box, seed, S, rmax, dt, corr in CALLS:
        radii = ic.log_radii(box / n, rmax, S)
        d32, d64 = parity.inputs(n, box, seed)
        d = d64 if dt == "c128" else d32
        ref_F, ref_I = _plan_path(d, n, box, radii, corr)
        dk = torch.from_numpy(d).cuda()
        F = torch.empty((n, n, n), dtype=torch.float32, device="cuda")
        I = torch.empty((n, n, n), dtype=torch.int32, device="cuda")
        torch.cuda.synchronize()
        pin.pin_collapse_times_noalloc(dk.data_ptr(), pin.PIN_C128 if dt == "c128" else pin.PIN_C64, n,
                                       box, radii, corr, F.data_ptr(), I.data_ptr(), stream.cuda_stream)
        stream.synchronize()
        st, wait_failed, counters = pin.pin_noalloc_status()
        assert st == pin.PIN_OK and wait_failed == 0, (st, wait_failed)
        assert counters[2] == 0, counters  # the FP64 redo queue never overflowed
        got_F, got_I = F.cpu().numpy().ravel(), I.cpu().numpy().ravel()
        # the same kernels and tables: bit for bit, which is within any tolerance
        assert np.array_equal(got_F, ref_F), (n, seed, int((got_F != ref_F).sum()))
        assert np.array_equal(got_I, ref_I), (n, seed, int((got_I != ref_I).sum()))
        assert (got_I >= 0).mean() > 0.05  # not vacuous: particles do collapse
        print("noalloc %d^3 seed %d %s corr %d: identical; redo counters %s" % (n, seed, dt, corr, counters))


def test_noalloc_rejects_sizes_beyond_its_workspace():
    import torch
    n = 96
    dk = torch.zeros((n, n, n // 2 + 1), dtype=torch.complex64, device="cuda")
    F = torch.empty((n, n, n), dtype=torch.float32, device="cuda")
    I = torch.empty((n, n, n), dtype=torch.int32, device="cuda")
    with pytest.raises(pin.PinError) as e:
        pin.pin_collapse_times_noalloc(dk.data_ptr(), pin.PIN_C64, n, 192.0, [4.0], 1,
                                       F.data_ptr(), I.data_ptr())
    assert e.value.status == pin.PIN_EINVAL
    # more radii than the static tables hold
    with pytest.raises(pin.PinError) as e:
        pin.pin_collapse_times_noalloc(dk.data_ptr(), pin.PIN_C64, 16, 32.0, np.full(65, 2.0), 1,
                                       F.data_ptr(), I.data_ptr())
    assert e.value.status == pin.PIN_EINVAL
