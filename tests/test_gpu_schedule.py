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


def test_set_radii_matches_fresh_plans():
    """pin_set_radii: one plan serves radius lists of other lengths and values
    (its graphs are kept per radius count) with the results of a plan made for
    each list, bit for bit."""
    import torch
    from paper_1305_1505_gb300 import pin
    n, box = 64, 128.0
    d32, _ = parity.inputs(n, box, 17)
    lists = [ic.log_radii(2.0, 30.0, 6), ic.log_radii(3.0, 20.0, 9), ic.log_radii(2.5, 25.0, 6)]
    fresh = []
    for radii in lists:
        p = pin.Plan(n, box, radii)
        p.set_ic(torch.from_numpy(d32).cuda())
        F, I = p.collapse_times()
        fresh.append((F.clone(), I.clone()))
        p.close()
    plan = pin.Plan(n, box, lists[0])
    plan.set_ic(torch.from_numpy(d32).cuda())
    for k in (0, 1, 2, 1, 0):
        plan.set_radii(lists[k])
        F, I = plan.collapse_times()
        assert torch.equal(F, fresh[k][0]) and torch.equal(I, fresh[k][1]), k
        h = plan.hessian(len(lists[k]) - 1)  # the scale index refers to the new list
        assert h.shape[0] == 6
    with pytest.raises(pin.PinError) as e:
        plan.set_radii(np.full(65, 2.0))
    assert e.value.status == pin.PIN_EINVAL
    with pytest.raises(pin.PinError) as e:
        plan.set_radii([2.0, -1.0])
    assert e.value.status == pin.PIN_EINVAL
    plan.close()
