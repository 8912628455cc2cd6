"""v_max (Sec. 2.1.1): the displacement of the field smoothed on R_max,
against the oracle, and F_max / scale index unchanged by the extra fields."""
import numpy as np
import pytest

import oracle
from paper_1305_1505_gb300 import ic
from tests import parity

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n,box,S", [(32, 64.0, 6), (48, 96.0, 5), (128, 512.0, 8)])
def test_vmax_parity(n, box, S):
    import torch
    from paper_1305_1505_gb300 import pin
    radii = ic.log_radii(4.0 * box / n, box / 5, S)
    d32, d64 = parity.inputs(n, box, 41)
    plan = pin.Plan(n, box, radii, velocities=True)
    plan.set_ic(torch.from_numpy(d32).cuda())
    F, I = plan.collapse_times()
    v = plan.velocities().cpu().numpy().reshape(3, -1).astype(np.float64)
    F, I = F.cpu().numpy().ravel(), I.cpu().numpy().ravel()
    orc = oracle.collapse_times(d64, box, radii, velocities=True, keep_all=n <= 48)
    parity.assert_parity(F, I, orc, d64, box, radii, label="v_max %d^3" % n)
    same = I == orc["idx"]
    vo = orc["vmax"]
    for c in range(3):
        rms = np.sqrt(np.mean(vo[c] ** 2))
        assert np.abs(v[c][same] - vo[c][same]).max() < 2e-5 * rms, c
    assert np.all(v[:, I < 0] == 0)
    # the plain mode gives the same F_max and index bit for bit
    plain = pin.Plan(n, box, radii)
    plain.set_ic(torch.from_numpy(d32).cuda())
    F2, I2 = plain.collapse_times()
    assert np.array_equal(F2.cpu().numpy().ravel(), F) and np.array_equal(I2.cpu().numpy().ravel(), I)


def test_velocities_need_the_mode():
    import torch
    from paper_1305_1505_gb300 import pin
    plan = pin.Plan(16, 32.0, [4.0])
    plan.set_ic(torch.zeros((16, 16, 9), dtype=torch.complex64, device="cuda"))
    plan.collapse_times()
    with pytest.raises(pin.PinError) as e:
        plan.velocities()
    assert e.value.status == pin.PIN_EINVAL
