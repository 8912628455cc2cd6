"""Radius schedules (pin_set_schedule): the overlapped schedules run the z
pass of one radius beside the x (and y) passes of the next on two streams,
and must give the serial schedule's results bit for bit."""
import numpy as np
import pytest

from paper_1305_1505_gb300 import ic
from tests import parity

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("vel", [False, True], ids=["plain", "velocities"])
def test_schedules_are_bit_identical(vel):
    import torch
    from paper_1305_1505_gb300 import pin
    n, box = 384, 1536.0
    radii = ic.log_radii(4.0, 120.0, 7)
    d32, _ = parity.inputs(n, box, 3)
    plan = pin.Plan(n, box, radii, stream=torch.cuda.Stream(), velocities=vel)
    plan.set_ic(torch.from_numpy(d32).cuda())
    out = {}
    for sched in (0, 1, 2, 0):
        pin.pin_set_schedule(plan.handle, sched)
        assert pin.pin_get_schedule(plan.handle) == sched
        for tiles in pin.pin_tile_options(n):
            plan.set_tiles(tiles, tiles)
            F, I = plan.collapse_times()
            got = [F.clone(), I.clone()] + ([plan.velocities()] if vel else [])
            if "ref" not in out:
                out["ref"] = got
                assert (I >= 0).float().mean() > 0.05
            else:
                for a, b in zip(out["ref"], got):
                    assert torch.equal(a, b), (sched, tiles)
    plan.close()


def test_overlapped_schedule_needs_a_fused_z_pass():
    import torch
    from paper_1305_1505_gb300 import pin
    plan = pin.Plan(64, 128.0, [4.0, 2.0])
    with pytest.raises(pin.PinError) as e:
        pin.pin_set_schedule(plan.handle, 1)
    assert e.value.status == pin.PIN_EINVAL
    assert pin.pin_get_schedule(plan.handle) == 0
    plan.close()
