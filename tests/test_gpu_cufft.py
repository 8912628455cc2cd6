"""Cross-check of the CUDA path's filter and line transforms against cuFFT
(torch.fft in double precision) at every supported grid size and on
non-cubic grids.  cuFFT is only the checker here: the fields come from
`pin_hessian` and `pin_displacements`, and are compared with
  phi_ij = IDFT[(k_i k_j / k^2) W(kR) delta(k)]   (Sec. 2.1.1, Hessian),
  psi_i  = IDFT[i k_i / k^2 delta(k)]             (Zel'dovich displacement),
computed by cuFFT's complex-to-real transform with the inverse convention of
the method (1/N^3 on the inverse), the Gaussian window W = exp(-k^2 R^2 / 2),
k = 0 removed, and the odd factors k_i zero where their index is the Nyquist
one (off-diagonal components and displacements), as in the readings of the
filter; and the trace rule phi_xx + phi_yy + phi_zz = IDFT(W delta) within
1e-5 of its rms."""
import math

import numpy as np
import pytest

from paper_1305_1505_gb300 import ic

pytestmark = pytest.mark.gpu

SIZES = [8, 16, 32, 48, 64, 96, 128, 192, 256, 384, 512, 768]
PAIRS = [(0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2)]


def _wavenumbers(shape, box):
    """Per-axis k (float64, on the device) of the half-spectrum grid and the
    masks of the Nyquist indices; cells are cubic, box is the side along x."""
    import torch
    nx, ny, nz = shape
    ks, nyq = [], []
    for a, n in enumerate((nx, ny, nz)):
        L = box * n / nx
        if a < 2:
            m = torch.fft.fftfreq(n, 1.0 / n, dtype=torch.float64, device="cuda")
        else:
            m = torch.arange(n // 2 + 1, dtype=torch.float64, device="cuda")
        view = [1, 1, 1]
        view[a] = -1
        ks.append((2 * math.pi / L * m).view(view))
        nyq.append((m.abs() == n // 2).view(view))
    return ks, nyq


def _cufft_fields(d, shape, box, R):
    """Six Hessian components (xx, yy, zz, xy, xz, yz) at radius R and the
    three unsmoothed displacement components, FP64 through cuFFT."""
    import torch
    ks, nyq = _wavenumbers(shape, box)
    k2 = ks[0] ** 2 + ks[1] ** 2 + ks[2] ** 2
    zero = k2 == 0
    inv = torch.where(zero, torch.zeros_like(k2), 1.0 / torch.where(zero, torch.ones_like(k2), k2))
    w = torch.exp(-0.5 * k2 * R * R)
    hs = []
    for i, j in PAIRS:
        t = ks[i] * ks[j] * inv * w * d
        if i != j:
            t = torch.where(nyq[i] | nyq[j], torch.zeros_like(t), t)
        hs.append(torch.fft.irfftn(t, s=shape))
    ps = []
    for i in range(3):
        t = 1j * ks[i] * inv * d
        t = torch.where(nyq[i], torch.zeros_like(t), t)
        ps.append(torch.fft.irfftn(t, s=shape))
    return torch.stack(hs), torch.stack(ps)


def _white(shape, seed):
    """Hermitian half-spectrum of unit white noise (every mode excited)."""
    import torch
    g = torch.Generator(device="cpu").manual_seed(seed)
    x = torch.randn(shape, generator=g, dtype=torch.float64)
    return torch.fft.rfftn(x).to("cuda")


def _check(shape, box, d64_dev, radii, label):
    import torch
    from paper_1305_1505_gb300 import pin
    plan = pin.Plan(shape, box, radii)
    try:
        plan.set_ic(d64_dev.to(torch.complex64))
        # the path sees the FP32 spectrum: the checker transforms the same values
        d = d64_dev.to(torch.complex64).to(torch.complex128)
        ks, _ = _wavenumbers(shape, box)
        k2 = ks[0] ** 2 + ks[1] ** 2 + ks[2] ** 2
        for s, R in enumerate(radii):
            h = plan.hessian(s).double()
            ref, psi_ref = _cufft_fields(d, shape, box, R)
            rms = float(ref.pow(2).mean().sqrt())
            err = float((h - ref).abs().max())
            assert err < 2e-5 * rms, "%s R=%g: max |phi - cuFFT| = %.3g (rms %.3g)" % (label, R, err, rms)
            # trace rule: phi_xx + phi_yy + phi_zz = IDFT(W delta) with k = 0 removed
            wd = torch.exp(-0.5 * k2 * R * R) * torch.where(k2 == 0, torch.zeros_like(d), d)
            tr_ref = torch.fft.irfftn(wd, s=shape)
            trms = float(tr_ref.pow(2).mean().sqrt())
            terr = float((h[0] + h[1] + h[2] - tr_ref).abs().max())
            assert terr < 1e-5 * trms, "%s R=%g: trace off by %.3g (rms %.3g)" % (label, R, terr, trms)
        psi = plan.displacements().double()
        prms = float(psi_ref.pow(2).mean().sqrt())
        perr = float((psi - psi_ref).abs().max())
        assert perr < 2e-5 * prms, "%s: max |psi - cuFFT| = %.3g (rms %.3g)" % (label, perr, prms)
    finally:
        plan.close()


@pytest.mark.parametrize("n", SIZES)
def test_cubic_against_cufft(n):
    """Seeded BBKS field of the benchmark's cells (4 Mpc/h), radii of two
    and of zero cells."""
    import torch
    box = 4.0 * n
    d = torch.from_numpy(ic.delta_k(n, box, 11, dtype=np.complex128)).cuda()
    _check((n, n, n), box, d, [8.0, 0.0], "%d^3" % n)


@pytest.mark.parametrize("shape", [(32, 48, 64), (64, 32, 16), (96, 16, 48)])
def test_non_cubic_against_cufft(shape):
    box = 2.0 * shape[0]
    _check(shape, box, _white(shape, 5), [3.0, 0.0], "x".join(map(str, shape)))
