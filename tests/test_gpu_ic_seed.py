"""delta(k) generated on the device (pin_set_ic_seed) against the host input
module's FP32 field: the same generator, up to the last bits of the device's
FP64 math functions."""
import numpy as np
import pytest

from paper_1305_1505_gb300 import ic

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n,box,seed", [(32, 64.0, 5), (48, 96.0, 6), (128, 512.0, 3)])
def test_seeded_field_equals_host_generator(n, box, seed):
    import torch
    from paper_1305_1505_gb300 import pin
    radii = ic.log_radii(2.0 * box / n, box / 5, 4)
    a = pin.Plan(n, box, radii)
    a.set_ic(torch.from_numpy(ic.delta_k(n, box, seed, dtype=np.complex64)).cuda())
    b = pin.Plan(n, box, radii)
    b.set_ic_seed(seed)
    # the deformation tensor at R = 0 (via the displacement) and at the first radius
    pa, pb = a.displacements().cpu().numpy(), b.displacements().cpu().numpy()
    ha, hb = a.hessian(0).cpu().numpy(), b.hessian(0).cpu().numpy()
    for x, y in ((pa, pb), (ha, hb)):
        same = np.mean(x == y)
        assert same > 0.999 and np.abs(x - y).max() <= 1e-5 * np.abs(x).max(), (same, np.abs(x - y).max())
    Fa, Ia = a.collapse_times()
    Fb, Ib = b.collapse_times()
    assert np.mean((Fa == Fb).cpu().numpy()) > 0.999 and np.mean((Ia == Ib).cpu().numpy()) > 0.9999
    a.close()
    b.close()


def test_seeded_batch_is_consecutive_seeds():
    import torch
    from paper_1305_1505_gb300 import pin
    n, box, radii = 32, 64.0, ic.log_radii(2.0, 12.0, 3)
    bplan = pin.Plan(n, box, radii, batch=3)
    bplan.set_ic_seed(40)
    Fb, Ib = bplan.collapse_times()
    for i in range(3):
        s = pin.Plan(n, box, radii)
        s.set_ic_seed(40 + i)
        F, I = s.collapse_times()
        assert torch.equal(F, Fb[i]) and torch.equal(I, Ib[i])
        s.close()
    bplan.close()


def test_seeded_field_needs_a_cubic_grid():
    from paper_1305_1505_gb300 import pin
    plan = pin.Plan((32, 16, 32), 64.0, [4.0])
    with pytest.raises(pin.PinError) as e:
        plan.set_ic_seed(1)
    assert e.value.status == pin.PIN_EINVAL
    plan.close()
