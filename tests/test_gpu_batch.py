"""Batched plans: B realisations in one launch per pass give, bit for bit,
what B single-realisation plans give (and those match the oracle in
test_gpu_parity)."""
import numpy as np
import pytest

from paper_1305_1505_gb300 import ic
from tests import parity

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n,box,B,S", [(32, 64.0, 3, 6), (128, 256.0, 2, 5), (384, 1536.0, 2, 3)])
def test_batch_matches_single_plans(n, box, B, S):
    import torch
    from paper_1305_1505_gb300 import pin
    radii = ic.log_radii(2.0 * box / n, 40.0, S)
    seeds = [100 + i for i in range(B)]
    fields = [ic.delta_k(n, box, s, dtype=np.complex64) for s in seeds]
    bplan = pin.Plan(n, box, radii, batch=B)
    bplan.set_ic(torch.from_numpy(np.stack(fields)).cuda())
    Fb, Ib = bplan.collapse_times()
    Fb, Ib = Fb.cpu().numpy(), Ib.cpu().numpy()
    bplan.close()
    splan = pin.Plan(n, box, radii)
    for i, d in enumerate(fields):
        splan.set_ic(torch.from_numpy(d).cuda())
        F, I = splan.collapse_times()
        assert np.array_equal(F.cpu().numpy(), Fb[i]), i
        assert np.array_equal(I.cpu().numpy(), Ib[i]), i
    splan.close()


def test_batch_against_oracle_small():
    import torch
    import oracle
    from paper_1305_1505_gb300 import pin
    n, box, S = 16, 64.0, 5
    radii = ic.log_radii(4.0, 16.0, S)
    d0, d0_64 = parity.inputs(n, box, 31)
    d1, d1_64 = parity.inputs(n, box, 32)
    plan = pin.Plan(n, box, radii, batch=2)
    plan.set_ic(np.stack([d0, d1]))
    F, I = plan.collapse_times()
    F, I = F.cpu().numpy(), I.cpu().numpy()
    for b, d64 in enumerate((d0_64, d1_64)):
        orc = oracle.collapse_times(d64, box, radii, keep_all=True)
        parity.assert_parity(F[b], I[b], orc, d64, box, radii, label="batch %d" % b)


def test_batch_rejects_tensor_dumps():
    from paper_1305_1505_gb300 import pin
    plan = pin.Plan(16, 64.0, [4.0], batch=2)
    import torch
    plan.set_ic(torch.zeros((2, 16, 16, 9), dtype=torch.complex64, device="cuda"))
    with pytest.raises(pin.PinError) as e:
        plan.hessian(0)
    assert e.value.status == pin.PIN_EINVAL
