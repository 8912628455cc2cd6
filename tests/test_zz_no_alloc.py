"""The no-allocation entry point (pin_collapse_times_noalloc) against
pin_collapse_times, through the C-ABI, on two calls in a row.

It exists for callers that cannot allocate device memory at call time (a
serving pool that already owns the device's memory, allocator hooks,
latency-critical code that cannot afford cudaFree's device-wide sync); its
workspace is a static device array shared by all calls, so the second call
also shows that nothing of the first call's contents leaks into it.  This file
sorts last so that a run stopping at its first failure has run everything
else already."""
import numpy as np
import pytest

from paper_1305_1505_gb300 import ic, pin
from tests import parity

pytestmark = pytest.mark.gpu


def _reference(d32, n, box, radii):
    import torch
    plan = pin.Plan(n, box, radii)
    plan.set_ic(torch.from_numpy(d32).cuda())
    F, I = plan.collapse_times()
    out = F.cpu().numpy().ravel(), I.cpu().numpy().ravel()
    plan.close()
    return out


def test_noalloc_matches_plan_path_two_calls():
    import torch
    n, box = 64, 100.0
    radii = ic.log_radii(box / n, 15.0, 20)
    stream = torch.cuda.Stream()
    F = torch.empty((n, n, n), dtype=torch.float32, device="cuda")
    I = torch.empty((n, n, n), dtype=torch.int32, device="cuda")
    for seed in (1, 2):  # two calls in a row, different inputs
        d32, _ = parity.inputs(n, box, seed)
        ref_F, ref_I = _reference(d32, n, box, radii)
        dk = torch.from_numpy(d32).cuda()
        torch.cuda.synchronize()
        pin.pin_collapse_times_noalloc(dk.data_ptr(), pin.PIN_C64, n, box, radii,
                                       pin.PIN_CORR_SPHERE, F.data_ptr(), I.data_ptr(),
                                       stream.cuda_stream)
        stream.synchronize()
        got_F = F.cpu().numpy().ravel()
        got_I = I.cpu().numpy().ravel()
        bad, rep = parity.classify(got_F, got_I, ref_F, ref_I)
        assert rep["f_bad"] == 0, rep
        assert rep["idx_mismatch"] <= max(1, 1e-4 * n ** 3), rep


def test_noalloc_rejects_grids_beyond_its_workspace():
    import torch
    n = 96
    dk = torch.zeros((n, n, n // 2 + 1), dtype=torch.complex64, device="cuda")
    F = torch.empty((n, n, n), dtype=torch.float32, device="cuda")
    I = torch.empty((n, n, n), dtype=torch.int32, device="cuda")
    with pytest.raises(pin.PinError) as e:
        pin.pin_collapse_times_noalloc(dk.data_ptr(), pin.PIN_C64, n, 192.0, [4.0], 1,
                                       F.data_ptr(), I.data_ptr())
    assert e.value.status == pin.PIN_EINVAL
