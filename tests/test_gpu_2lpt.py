"""Second-order LPT displacement on the GPU against the oracle (which is
pinned to the closed form of two crossed waves on the CPU)."""
import numpy as np
import pytest

import oracle
from paper_1305_1505_gb300 import ic
from tests import parity

pytestmark = pytest.mark.gpu

TOL = 5e-5  # of the rms of each component


@pytest.mark.parametrize("n,box", [(32, 64.0), (48, 96.0), (64, 100.0), (128, 512.0)])
def test_2lpt_matches_oracle(n, box):
    import torch
    from paper_1305_1505_gb300 import pin
    d32, d64 = parity.inputs(n, box, 71)
    plan = pin.Plan(n, box, ic.log_radii(2.0 * box / n, box / 4, 4))
    plan.set_ic(torch.from_numpy(d32).cuda())
    F0, I0 = plan.collapse_times()
    F0, I0 = F0.cpu().numpy(), I0.cpu().numpy()
    psi2 = plan.displacements_2lpt().double().cpu().numpy()
    ref = oracle.displacement_2lpt(d64, box)
    for c in range(3):
        rms = np.sqrt(np.mean(ref[c] ** 2))
        err = np.abs(psi2[c] - ref[c]).max()
        assert err <= TOL * rms, (c, err / rms)
    # host output is the device output
    h = np.empty((3, n, n, n), dtype=np.float32)
    pin.pin_displacements_2lpt(plan.handle, h.ctypes.data, 0)
    assert np.array_equal(h, psi2.astype(np.float32))
    # the collapse state survives, and the next collapse call is unaffected
    F1, I1 = plan.collapse_times()
    assert np.array_equal(F1.cpu().numpy(), F0) and np.array_equal(I1.cpu().numpy(), I0)
    plan.close()


def test_2lpt_two_crossed_waves_on_gpu():
    import torch
    from paper_1305_1505_gb300 import pin
    n, box = 64, 128.0
    x = np.arange(n) * box / n
    X, Y, Z = np.meshgrid(x, x, x, indexing="ij")
    k1, k2 = 2 * np.pi * 3 / box, 2 * np.pi * 5 / box
    A, B = 0.6, 0.9
    dk = np.fft.rfftn(A * np.cos(k1 * X) + B * np.cos(k2 * Y)).astype(np.complex64)
    plan = pin.Plan(n, box, [4.0])
    plan.set_ic(torch.from_numpy(dk).cuda())
    psi2 = plan.displacements_2lpt().double().cpu().numpy()
    K2 = k1 ** 2 + k2 ** 2
    sp, sm = np.sin(k1 * X + k2 * Y), np.sin(k1 * X - k2 * Y)
    c = -(3.0 / 7.0) * A * B / 2 / K2
    amp = abs(c) * max(k1, k2) * 2
    assert np.abs(psi2[0] - c * k1 * (sp + sm)).max() < 2e-5 * amp
    assert np.abs(psi2[1] - c * k2 * (sp - sm)).max() < 2e-5 * amp
    assert np.abs(psi2[2]).max() < 2e-5 * amp
    plan.close()
