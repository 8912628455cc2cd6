"""Failure paths of the C-ABI, made to fire without any GPU fault: a host
deadline that expires while the device works (PIN_ETIMEOUT), device waits
whose budget is set so small that they run out (the kernels give up, record
the error and return; the host reads PIN_ECUDA once and the plan stays
usable), and a device allocation made to fail on the host (PIN_ENOMEM with
nothing left allocated)."""
import numpy as np
import pytest

from paper_1305_1505_gb300 import ic
from tests import parity

pytestmark = pytest.mark.gpu


def test_sync_deadline_expires_then_work_completes():
    import torch
    from paper_1305_1505_gb300 import pin
    n, box = 384, 1536.0
    radii = ic.log_radii(4.0, 120.0, 12)
    plan = pin.Plan(n, box, radii, stream=torch.cuda.Stream())
    d32, _ = parity.inputs(n, box, 3)
    plan.set_ic(torch.from_numpy(d32).cuda())
    F, I = plan.collapse_times()  # first call: builds the graph
    ref = F.clone(), I.clone()
    plan.collapse_times(F, I, sync=False)
    st = pin.pin_sync(plan.handle, 1000)  # 1 us: the 12-radius loop takes milliseconds
    assert st == pin.PIN_ETIMEOUT, pin.pin_strerror(st)
    assert pin.pin_sync(plan.handle, -1) == pin.PIN_OK
    assert torch.equal(F, ref[0]) and torch.equal(I, ref[1])


def test_transfer_waits_run_out_and_the_plan_recovers():
    import torch
    from paper_1305_1505_gb300 import pin
    n, box = 128, 512.0
    radii = ic.log_radii(4.0, 60.0, 6)
    d32, _ = parity.inputs(n, box, 7)
    plan = pin.Plan(n, box, radii, stream=torch.cuda.Stream())
    plan.set_ic(torch.from_numpy(d32).cuda())
    F0, I0 = plan.collapse_times()
    F0, I0 = F0.clone(), I0.clone()
    # a budget of one clock: the first wait for a staged tile runs out
    pin.pin_set_wait_budget(plan.handle, 1)
    F, I = plan.collapse_times(sync=False)
    st = pin.pin_sync(plan.handle, -1)
    assert st == pin.PIN_ECUDA, pin.pin_strerror(st)
    assert "timed out" in pin.pin_last_error(plan.handle)
    assert pin.pin_sync(plan.handle, -1) == pin.PIN_OK  # reported once
    # the default budget again: the same plan gives the reference bits
    pin.pin_set_wait_budget(plan.handle, 0)
    F, I = plan.collapse_times()
    assert torch.equal(F, F0) and torch.equal(I, I0)
    with pytest.raises(pin.PinError) as e:
        pin.pin_set_wait_budget(plan.handle, -5)
    assert e.value.status == pin.PIN_EINVAL


def test_injected_allocation_failure_leaves_nothing_allocated():
    import torch
    from paper_1305_1505_gb300 import pin
    n, box = 64, 128.0
    stream = torch.cuda.Stream()
    torch.cuda.synchronize()
    try:
        for vel in (False, True):
            # the plan's device arrays: Phi0, U, V, [psi, v state,] F_max, index,
            # multipliers, twiddles, counters, redo queue, its count, error word
            allocs = 13 if vel else 11
            for nth in range(allocs):
                free0, _ = torch.cuda.mem_get_info()
                pin.pin_debug_fail_alloc(nth)
                with pytest.raises(pin.PinError) as e:
                    pin.Plan(n, box, [8.0, 4.0], stream=stream, velocities=vel)
                assert e.value.status == pin.PIN_ENOMEM, (vel, nth)
                free1, _ = torch.cuda.mem_get_info()
                assert free1 == free0, (vel, nth, free0 - free1)
            # one past the last allocation: the injection is not reached and the
            # plan is made; the pending injection is then cancelled
            pin.pin_debug_fail_alloc(allocs)
            plan = pin.Plan(n, box, [8.0, 4.0], stream=stream, velocities=vel)
            pin.pin_debug_fail_alloc(-1)
            plan.set_ic(torch.from_numpy(parity.inputs(n, box, 9)[0]).cuda())
            F, I = plan.collapse_times()
            assert (I >= 0).float().mean() > 0.05
            plan.close()
    finally:
        pin.pin_debug_fail_alloc(-1)
