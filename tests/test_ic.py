"""The seeded input generator (CPU): determinism, Hermitian symmetry and the
sigma8 normalisation of Sec. 2.1.1, checked against independent routines."""
import numpy as np
import pytest

from paper_1305_1505_gb300 import ic


def test_splitmix64_reference_values():
    # splitmix64 with state 0: the first outputs of the published generator
    # (Steele, Lea & Flood 2014; the stream java.util.SplittableRandom and
    # Vigna's splitmix64.c produce for seed 0).
    assert ic.splitmix64(0) == 0xE220A8397B1DCDAF
    assert ic.splitmix64(0x9E3779B97F4A7C15) == 0x6E789E6AA1B965F4


def test_deterministic_and_seed_dependent():
    a = ic.delta_k(16, 100.0, 1, dtype=np.complex128)
    b = ic.delta_k(16, 100.0, 1, dtype=np.complex128)
    c = ic.delta_k(16, 100.0, 2, dtype=np.complex128)
    assert np.array_equal(a.view(np.uint64), b.view(np.uint64))
    assert not np.allclose(a, c)
    f = ic.delta_k(16, 100.0, 1, dtype=np.complex64)
    assert np.array_equal(f, a.astype(np.complex64))


@pytest.mark.parametrize("n", [8, 12, 16])
def test_hermitian_planes_and_zero_mode(n):
    d = ic.delta_k(n, 64.0, 3, dtype=np.complex128)
    assert d[0, 0, 0] == 0
    for iz in (0, n // 2):
        plane = d[:, :, iz]
        mirror = np.conj(plane[(-np.arange(n)) % n][:, (-np.arange(n)) % n])
        assert np.array_equal(plane, mirror)
    # the field is real: numpy's irfftn of it round-trips through rfftn
    f = np.fft.irfftn(d, s=(n, n, n), axes=(0, 1, 2))
    assert np.allclose(np.fft.rfftn(f, axes=(0, 1, 2)), d, atol=1e-9 * np.abs(d).max())


def test_amplitude_matches_quadrature():
    scipy = pytest.importorskip("scipy.integrate")
    amp = ic.amplitude()

    def integrand(lnk):
        k = np.exp(lnk)
        x = 8.0 * k
        w = 3 * (np.sin(x) - x * np.cos(x)) / x ** 3
        return ic.power(k, amp=amp)[0] * w * w * k ** 3 / (2 * np.pi ** 2)

    val, _ = scipy.quad(integrand, np.log(1e-5), np.log(1e3), limit=400)
    assert abs(np.sqrt(val) - 0.8) < 1e-6


def test_bbks_limits():
    assert ic.bbks(0.0) == 1.0
    assert abs(ic.bbks(1e-6) - 1.0) < 1e-4
    # large-q tail ~ ln(2.34 q) / (2.34 q) / (6.71 q)
    q = 1e4
    assert abs(ic.bbks(q) / (np.log(2.34 * q) / (2.34 * q) / (6.71 * q)) - 1) < 1e-2


def test_measured_spectrum_matches_input():
    """Shell-averaged |delta(k)|^2 L^3 / N^6 recovers P(k) within sampling error."""
    n, box = 64, 256.0
    d = ic.delta_k(n, box, 5, dtype=np.complex128)
    amp = ic.amplitude()
    kf = 2 * np.pi / box
    m = np.fft.fftfreq(n, 1.0 / n)
    mz = np.arange(n // 2 + 1)
    kk = kf * np.sqrt(m[:, None, None] ** 2 + m[None, :, None] ** 2 + mz[None, None, :] ** 2)
    pk = np.abs(d) ** 2 * box ** 3 / float(n) ** 6
    wgt = np.where((mz == 0) | (mz == n // 2), 1.0, 2.0)[None, None, :] * np.ones_like(kk)
    edges = np.linspace(4 * kf, 24 * kf, 6)
    for lo, hi in zip(edges[:-1], edges[1:]):
        sel = (kk >= lo) & (kk < hi)
        meas = np.sum(pk[sel] * wgt[sel]) / np.sum(wgt[sel])
        pred = np.sum(ic.power(kk[sel][::50], amp=amp)) / kk[sel][::50].size
        nmodes = np.sum(wgt[sel])
        assert abs(meas / pred - 1) < 6 / np.sqrt(nmodes) + 0.05


def test_log_radii_largest_first():
    r = ic.log_radii(1.5625, 15.0, 20)
    assert r.size == 20 and abs(r[0] - 15.0) < 1e-12 and abs(r[-1] - 1.5625) < 1e-12
    assert np.all(np.diff(r) < 0)
