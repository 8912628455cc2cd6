"""Non-cubic grids (the paper's code runs on them as well, Sec. 2.1.1): the
CUDA path on nx x ny x nz grids with cubic cells against the oracle."""
import numpy as np
import pytest

import oracle
from paper_1305_1505_gb300 import ic
from tests import parity

pytestmark = pytest.mark.gpu

SHAPES = [(32, 48, 64), (64, 32, 16), (16, 64, 32)]


def _field(shape, box, seed):
    """Gaussian field with the BBKS spectrum of the cubic inputs on an
    nx x ny x nz grid of cubic cells (side box along x): numpy's rfftn of
    white noise times sqrt(P(k) nx ny nz / V)."""
    nx, ny, nz = shape
    L = [box, box * ny / nx, box * nz / nx]
    V = L[0] * L[1] * L[2]
    w = np.fft.rfftn(np.random.default_rng(seed).normal(size=shape))
    kx = 2 * np.pi * np.fft.fftfreq(nx, 1.0 / nx) / L[0]
    ky = 2 * np.pi * np.fft.fftfreq(ny, 1.0 / ny) / L[1]
    kz = 2 * np.pi * np.arange(nz // 2 + 1) / L[2]
    k = np.sqrt(kx[:, None, None] ** 2 + ky[None, :, None] ** 2 + kz[None, None, :] ** 2)
    ku, inv = np.unique(k.ravel(), return_inverse=True)
    Pu = np.zeros(ku.size)
    Pu[ku > 0] = ic.power(ku[ku > 0])
    P = Pu[inv].reshape(k.shape)
    d = w * np.sqrt(P * nx * ny * nz / V)
    d[0, 0, 0] = 0.0
    return d.astype(np.complex64), d.astype(np.complex64).astype(np.complex128)


@pytest.mark.parametrize("shape", SHAPES)
def test_non_cubic_collapse_hessian_displacement(shape):
    import torch
    from paper_1305_1505_gb300 import pin
    box = 2.0 * shape[0]
    # radii up to a quarter of the shortest side: a radius comparable to a box
    # side smooths away all structure along it, leaving one eigenvalue at
    # zero to within FP32 rounding of the others, where F ~ lambda^(1/3)
    # cannot be resolved in FP32 (outside the method's range)
    radii = ic.log_radii(2.0, box * min(shape) / shape[0] / 4, 6)
    d32, d64 = _field(shape, box, 81)
    plan = pin.Plan(shape, box, radii, velocities=True)
    plan.set_ic(torch.from_numpy(d32).cuda())
    F, I = plan.collapse_times()
    assert tuple(F.shape) == shape
    orc = oracle.collapse_times(d64, box, radii, keep_all=True, velocities=True)
    Fh, Ih = F.cpu().numpy().ravel(), I.cpu().numpy().ravel()
    parity.assert_parity(Fh, Ih, orc, d64, box, radii, label=str(shape))
    # v_max: the displacement smoothed on R_max, where the indices agree
    v = plan.velocities().double().cpu().numpy().reshape(3, -1)
    same = I.cpu().numpy().ravel() == orc["idx"]
    vrms = np.sqrt(np.mean(orc["vmax"] ** 2))
    assert np.abs(v[:, same] - orc["vmax"][:, same]).max() < 2e-5 * vrms
    # the deformation tensor at one radius and the unsmoothed displacement
    h = plan.hessian(2).double().cpu().numpy()
    href, _ = oracle.hessian(d64, box, radii[2])
    assert np.abs(h - href).max() < 2e-5 * np.sqrt(np.mean(href ** 2))
    psi = plan.displacements().double().cpu().numpy()
    pref = oracle.displacement(d64, box, 0.0)
    assert np.abs(psi - pref).max() < 2e-5 * np.sqrt(np.mean(pref ** 2))
    # second-order displacement
    p2 = plan.displacements_2lpt().double().cpu().numpy()
    p2ref = oracle.displacement_2lpt(d64, box)
    for c in range(3):
        assert np.abs(p2[c] - p2ref[c]).max() < 5e-5 * np.sqrt(np.mean(p2ref[c] ** 2)), c
    plan.close()


def test_non_cubic_fragment_order():
    import torch
    from paper_1305_1505_gb300 import pin
    shape, box = (48, 32, 64), 96.0
    d32, _ = _field(shape, box, 82)
    plan = pin.Plan(shape, box, ic.log_radii(2.0, 8.0, 4))
    plan.set_ic(torch.from_numpy(d32).cuda())
    F, _ = plan.collapse_times()
    order, nb = plan.fragment_order()
    oref, nbref = oracle.fragment_order(F.cpu().numpy())
    assert np.array_equal(order.cpu().numpy(), oref)
    assert np.array_equal(nb.cpu().numpy().astype(np.int64), nbref)
    plan.close()



@pytest.mark.parametrize("shape", [(32, 32, 32), (64, 32, 16)])
def test_one_shot_helper_matches_plan(shape):
    """pin.collapse_times(delta_k, radii, box) reads the grid from the
    half-spectrum's shape and gives the plan's results bit for bit."""
    import torch
    from paper_1305_1505_gb300 import pin
    box = 2.0 * shape[0]
    radii = ic.log_radii(2.0, box * min(shape) / shape[0] / 4, 4)
    d32, _ = _field(shape, box, 83)
    dk = torch.from_numpy(d32).cuda()
    F1, I1 = pin.collapse_times(dk, radii, box)
    plan = pin.Plan(shape, box, radii)
    try:
        plan.set_ic(dk)
        F2, I2 = plan.collapse_times()
        assert tuple(F1.shape) == shape
        assert torch.equal(F1, F2) and torch.equal(I1, I2)
    finally:
        plan.close()
