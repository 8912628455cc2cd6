"""The all-FP64 precision mode (PIN_FP64) against the FP64 oracle: F_max
within 1e-10 (relative, with an absolute floor of 1e-10 of the rms), the
radius index equal except at near-ties, every particle outside that either
ill-conditioned in FP64 by the oracle's own measure (half-width 1e-12) or not
at all; radix-2, radix-3 and non-cubic grids, both correction modes."""
import numpy as np
import pytest

import oracle
from paper_1305_1505_gb300 import ic
from tests import parity

pytestmark = pytest.mark.gpu

REL64, U64 = 1e-10, 1e-12


@pytest.mark.parametrize("n,box,seed,S,corr", [(16, 64.0, 51, 6, 1), (32, 64.0, 52, 8, 1), (48, 96.0, 53, 8, 1),
                                               (64, 100.0, 1, 20, 1), (32, 64.0, 54, 6, 0)])
def test_fp64_mode_matches_the_oracle(n, box, seed, S, corr):
    import torch
    from paper_1305_1505_gb300 import pin
    radii = ic.log_radii(box / n, box / 6, S)
    d32, d64 = parity.inputs(n, box, seed)
    plan = pin.Plan(n, box, radii, correction=corr, precision=pin.PIN_FP64)
    plan.set_ic(torch.from_numpy(d64).cuda())  # C128 input: the oracle's own values
    F, I = plan.collapse_times_f64()
    orc = oracle.collapse_times(d64, box, radii, correction=corr, keep_all=True)
    rep = parity.assert_parity(F.cpu().numpy(), I.cpu().numpy(), orc, d64, box, radii, correction=corr,
                               label="fp64 %d^3" % n, rel=REL64, abs_frac=REL64, u=U64)
    assert rep["max_rel_err"] < 1e-8, rep
    # the FP32 output of the same plan is its FP64 result rounded
    F32, I32 = plan.collapse_times()
    assert torch.equal(F32.cpu(), F.cpu().float()) and torch.equal(I32.cpu(), I.cpu())
    plan.close()


def test_fp64_mode_non_cubic():
    import torch
    from paper_1305_1505_gb300 import pin
    from tests.test_gpu_noncubic import _field
    shape, box = (32, 48, 16), 64.0
    radii = ic.log_radii(2.0, 6.0, 5)
    _, d64 = _field(shape, box, 61)
    plan = pin.Plan(shape, box, radii, precision=pin.PIN_FP64)
    plan.set_ic(torch.from_numpy(d64).cuda())
    F, I = plan.collapse_times_f64()
    orc = oracle.collapse_times(d64, box, radii, keep_all=True)
    parity.assert_parity(F.cpu().numpy(), I.cpu().numpy(), orc, d64, box, radii, label="fp64 %s" % (shape,),
                         rel=REL64, abs_frac=REL64, u=U64)
    plan.close()


def test_fp64_mode_argument_checks():
    from paper_1305_1505_gb300 import pin
    with pytest.raises(pin.PinError) as e:
        pin.Plan(16, 32.0, [2.0], precision=pin.PIN_FP64, batch=2)
    assert e.value.status == pin.PIN_EINVAL
    plan = pin.Plan(16, 32.0, [2.0])
    import torch
    plan.set_ic(torch.zeros((16, 16, 9), dtype=torch.complex64, device="cuda"))
    with pytest.raises(pin.PinError) as e:
        plan.collapse_times_f64()
    assert e.value.status == pin.PIN_EINVAL
    plan.close()
