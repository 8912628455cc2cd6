"""Fragmentation front end (Sec. 2.1.2): the GPU order of the particles in
descending F_max and the count of neighbours that come before each one,
bit for bit against the oracle applied to the same (GPU) F_max field."""
import numpy as np
import pytest

import oracle
from paper_1305_1505_gb300 import ic
from tests import parity

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n,box,S", [(8, 32.0, 3), (32, 64.0, 6), (48, 96.0, 5), (64, 100.0, 8), (128, 512.0, 6)])
def test_fragment_order_matches_oracle(n, box, S):
    import torch
    from paper_1305_1505_gb300 import pin
    radii = ic.log_radii(2.0 * box / n, box / 4, S)
    d32, _ = parity.inputs(n, box, 61)
    plan = pin.Plan(n, box, radii)
    plan.set_ic(torch.from_numpy(d32).cuda())
    F, _ = plan.collapse_times()
    order, nb = plan.fragment_order()
    Fh = F.cpu().numpy()
    oref, nbref = oracle.fragment_order(Fh)
    assert np.array_equal(order.cpu().numpy(), oref)
    assert np.array_equal(nb.cpu().numpy().astype(np.int64), nbref)
    assert (Fh == 0).any()  # the ties at F = 0 (particles that never collapse) are exercised
    # host outputs are the device outputs
    oh = np.empty(n ** 3, dtype=np.int32)
    nh = np.empty((n, n, n), dtype=np.uint8)
    pin.pin_fragment_order(plan.handle, oh.ctypes.data, nh.ctypes.data, 0)
    assert np.array_equal(oh, oref) and np.array_equal(nh.astype(np.int64), nbref)
    # either output alone
    o_only, none = plan.fragment_order(n_before=False)
    assert none is None and np.array_equal(o_only.cpu().numpy(), oref)
    plan.close()


def test_fragment_order_all_ties():
    import torch
    from paper_1305_1505_gb300 import pin
    n = 32
    plan = pin.Plan(n, 64.0, [8.0, 4.0])
    plan.set_ic(torch.zeros((n, n, n // 2 + 1), dtype=torch.complex64, device="cuda"))
    F, I = plan.collapse_times()
    assert float(F.abs().max()) == 0.0
    order, nb = plan.fragment_order()
    assert np.array_equal(order.cpu().numpy(), np.arange(n ** 3))
    _, nbref = oracle.fragment_order(np.zeros((n, n, n), dtype=np.float32))
    assert np.array_equal(nb.cpu().numpy().astype(np.int64), nbref)
    plan.close()


def test_fragment_order_errors():
    import torch
    from paper_1305_1505_gb300 import pin
    plan = pin.Plan(16, 64.0, [4.0])
    plan.set_ic(torch.zeros((16, 16, 9), dtype=torch.complex64, device="cuda"))
    with pytest.raises(pin.PinError) as e:
        plan.fragment_order()
    assert e.value.status == pin.PIN_ESTATE
    plan.collapse_times()
    with pytest.raises(pin.PinError) as e:
        pin.pin_fragment_order(plan.handle, 0, 0, 1)
    assert e.value.status == pin.PIN_EINVAL
    plan.close()
    bplan = pin.Plan(16, 64.0, [4.0], batch=2)
    bplan.set_ic(torch.zeros((2, 16, 16, 9), dtype=torch.complex64, device="cuda"))
    bplan.collapse_times()
    with pytest.raises(pin.PinError) as e:
        bplan.fragment_order()
    assert e.value.status == pin.PIN_EINVAL
    bplan.close()
