"""Pins of the FP64 oracle to things other than itself (CPU only).

Each test checks the oracle against a closed form, a brute-force sum, a
library routine in a special case, or a textbook value, chosen so that a
dropped term, a wrong sign or index, or a transposed axis fails one of them.
"""
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_1305_1505_gb300 import ic

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    vals = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            k, v = line.split(None, 1)
            vals[k] = v
    return vals


# ---------------------------------------------------------------- DFT pins --

def _dft_matrix(n, sign):
    j = np.arange(n)
    return np.exp(sign * 2j * np.pi * np.outer(j, j) / n)


@pytest.mark.parametrize("n", [1, 2, 8, 16, 12, 6, 9])
def test_dft1d_matches_brute_force(n):
    rng = np.random.default_rng(n)
    x = rng.normal(size=n) + 1j * rng.normal(size=n)
    for sign in (+1, -1):
        ref = _dft_matrix(n, sign) @ x
        got = oracle.dft1d(x, sign)
        assert np.allclose(got, ref, rtol=0, atol=1e-12 * max(1, np.abs(ref).max()))
    # library special case: the unnormalised inverse DFT is n * numpy.fft.ifft
    assert np.allclose(oracle.dft1d(x, +1), n * np.fft.ifft(x), atol=1e-12 * n)


@pytest.mark.parametrize("n", [8, 6])
def test_idft3d_matches_brute_force(n):
    rng = np.random.default_rng(3)
    a = rng.normal(size=(n, n, n)) + 1j * rng.normal(size=(n, n, n))
    E = _dft_matrix(n, +1)
    ref = np.einsum("ai,bj,ck,ijk->abc", E, E, E, a) / n ** 3
    got = oracle.idft3d(a)
    assert np.abs(got - ref).max() < 1e-13 * np.abs(ref).max()


@pytest.mark.parametrize("n", [16, 12])
def test_parseval(n):
    rng = np.random.default_rng(5)
    a = rng.normal(size=(n, n, n)) + 1j * rng.normal(size=(n, n, n))
    f = oracle.idft3d(a)
    lhs = np.sum(np.abs(f) ** 2)
    rhs = np.sum(np.abs(a) ** 2) / n ** 3
    assert abs(lhs - rhs) < 1e-12 * rhs


# ------------------------------------------------------------- filter pins --

def _field(n, box, seed):
    return ic.delta_k(n, box, seed, dtype=np.complex128)


def test_hessian_is_real_for_hermitian_input():
    d = _field(16, 100.0, 11)
    h, max_imag = oracle.hessian(d, 100.0, 4.0)
    assert max_imag < 1e-13 * np.abs(h).max()


@pytest.mark.parametrize("n,box,radius", [(16, 100.0, 4.0), (12, 60.0, 3.0), (8, 50.0, 0.0)])
def test_trace_equals_smoothed_delta(n, box, radius):
    """phi_xx + phi_yy + phi_zz = IDFT(W delta): the filter's trace rule
    (del^2 phi = delta), against numpy's irfftn of the Gaussian-smoothed field.
    Nyquist modes are kept on the diagonal, so the rule is exact."""
    d = _field(n, box, 7)
    h, _ = oracle.hessian(d, box, radius)
    m = np.fft.fftfreq(n, 1.0 / n)
    m[n // 2] = -n // 2
    mz = np.arange(n // 2 + 1, dtype=float)
    mz[-1] = -n // 2
    kf = 2 * np.pi / box
    k2 = (kf * m[:, None, None]) ** 2 + (kf * m[None, :, None]) ** 2 + (kf * mz[None, None, :]) ** 2
    sm = d * np.exp(-0.5 * k2 * radius ** 2)
    sm[0, 0, 0] = 0.0
    ref = np.fft.irfftn(sm, s=(n, n, n), axes=(0, 1, 2))
    tr = h[0] + h[1] + h[2]
    assert np.abs(tr - ref).max() < 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("mode", [(1, 2, 3), (5, 1, 2), (3, 6, 1), (0, 0, 2), (4, 0, 0)])
def test_single_mode_closed_form(mode):
    """A single Fourier mode (plus its Hermitian mirror) gives
    phi_ij(q) = (k_i k_j / k^2) W(k) 2 Re(A e^{i k.q}) / n^3, which pins the
    sign convention, the axis order and the normalisation of every component."""
    n, box, radius = 8, 40.0, 2.0
    d = np.zeros((n, n, n // 2 + 1), dtype=np.complex128)
    amp = 0.7 - 1.3j
    mx, my, mz = mode
    d[mx, my, mz] = amp
    if mz == 0:
        d[(-mx) % n, (-my) % n, 0] = np.conj(amp)
    h, _ = oracle.hessian(d, box, radius)
    sx = mx if mx < n // 2 else mx - n
    sy = my if my < n // 2 else my - n
    sz = mz
    kf = 2 * np.pi / box
    k = np.array([kf * sx, kf * sy, kf * sz])
    k2 = k @ k
    q = np.indices((n, n, n))
    phase = 2 * np.pi * (sx * q[0] + sy * q[1] + sz * q[2]) / n
    wave = 2 * np.real(amp * np.exp(1j * phase)) / n ** 3
    if mz == 0 and (mx, my) == ((-mx) % n, (-my) % n):
        wave = wave / 2
    w = np.exp(-0.5 * k2 * radius ** 2)
    pairs = [(0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2)]
    for c, (i, j) in enumerate(pairs):
        ref = k[i] * k[j] / k2 * w * wave
        assert np.abs(h[c] - ref).max() < 1e-14 + 1e-12 * np.abs(wave).max(), (c, mode)


def test_offdiagonal_nyquist_is_zeroed():
    """A mode with k_x on the Nyquist index feeds xx, yy, zz, yz but never xy or
    xz (they would not be Hermitian)."""
    n, box = 8, 40.0
    d = np.zeros((n, n, n // 2 + 1), dtype=np.complex128)
    d[n // 2, 1, 2] = 1.0 + 0.5j
    h, _ = oracle.hessian(d, box, 1.0)
    assert np.abs(h[3]).max() == 0.0 and np.abs(h[4]).max() == 0.0
    assert np.abs(h[0]).max() > 0 and np.abs(h[5]).max() > 0


def test_direct_point_sum_matches_fft_path():
    """The direct sum over the half-spectrum at one point (a different
    algorithm) agrees with the FFT path."""
    n, box, radius = 12, 80.0, 5.0
    d = _field(n, box, 3)
    h, _ = oracle.hessian(d, box, radius)
    rng = np.random.default_rng(0)
    for _ in range(4):
        q = rng.integers(0, n, size=3)
        for c in range(6):
            v = oracle.hessian_point(d, box, radius, c, q)
            assert abs(v - h[c][tuple(q)]) < 1e-12 * np.abs(h[c]).max()


# -------------------------------------------------------- eigenvalue pins --

def _random_rotation(rng):
    q, r = np.linalg.qr(rng.normal(size=(3, 3)))
    return q * np.sign(np.diag(r))


def _h6(a):
    return np.array([a[0, 0], a[1, 1], a[2, 2], a[0, 1], a[0, 2], a[1, 2]])


@pytest.mark.parametrize("lam", [(3.0, -1.0, 0.5), (1.0, 1.0, -2.0), (2.0, 2.0, 2.0),
                                 (0.0, 0.0, 0.0), (1e-3, -5.0, 7.0), (4.0, 4.0 + 1e-9, 1.0)])
def test_eigen_rotated_diagonal(lam):
    rng = np.random.default_rng(1)
    for _ in range(5):
        Q = _random_rotation(rng)
        A = Q @ np.diag(lam) @ Q.T
        got = oracle.eig3(_h6(A))
        ref = np.sort(np.array(lam))[::-1]
        assert np.allclose(got, ref, rtol=0, atol=1e-13 * max(1.0, np.abs(ref).max()))


def test_eigen_characteristic_polynomial_residual():
    rng = np.random.default_rng(2)
    for _ in range(200):
        h = rng.normal(size=6)
        A = np.array([[h[0], h[3], h[4]], [h[3], h[1], h[5]], [h[4], h[5], h[2]]])
        lam = oracle.eig3(h)
        assert lam[0] >= lam[1] >= lam[2]
        for l in lam:
            assert abs(np.linalg.det(A - l * np.eye(3))) < 1e-12 * np.abs(A).max() ** 3
        assert abs(lam.sum() - np.trace(A)) < 1e-13 * np.abs(A).max() * 3


# ---------------------------------------------------------- collapse pins --

def _spherical_series_coeffs():
    """LPT radius series r/q = 1 - (k1 x + k2 x^2 + k3 x^3) of a sphere of
    linear contrast x, derived here by inverting 1 + delta_NL = (r/q)^-3 with
    the textbook vertices nu2, nu3 (Bernardeau 1994)."""
    g = _golden("spherical_collapse.txt")
    nu2 = Fraction(g["nu2"])
    nu3 = Fraction(g["nu3"])
    b, c = nu2 / 2, nu3 / 6  # delta_NL = x + b x^2 + c x^3
    # a = 1 - (1 + y)^(-1/3) = y/3 - 2/9 y^2 + 14/81 y^3 + O(y^4), y = delta_NL
    k1 = Fraction(1, 3)
    k2 = b / 3 - Fraction(2, 9)
    k3 = c / 3 - Fraction(4, 9) * b + Fraction(14, 81)
    return k1, k2, k3


def test_spherical_series_textbook_coefficients():
    k1, k2, k3 = _spherical_series_coeffs()
    assert (k1, k2, k3) == (Fraction(1, 3), Fraction(1, 21), Fraction(23, 1701))
    # the oracle's axis coefficients for a sphere of contrast delta reproduce them
    for delta in (0.3, 1.0, 2.5):
        lam = np.full(3, delta / 3)
        for i in range(3):
            c = oracle.axis_coeffs(lam, i)
            assert np.allclose(c, [float(k1) * delta, float(k2) * delta ** 2,
                                   float(k3) * delta ** 3], rtol=1e-14)


@pytest.mark.parametrize("delta", [0.05, 0.8, 1.686, 3.0, 10.0])
def test_sphere_uncorrected_is_series_root(delta):
    k1, k2, k3 = (float(v) for v in _spherical_series_coeffs())
    roots = np.roots([k3, k2, k1, -1.0])
    x3 = min(r.real for r in roots if abs(r.imag) < 1e-12 and r.real > 0)
    assert abs(oracle.x3() - x3) < 1e-13
    h6 = np.array([delta / 3] * 3 + [0.0] * 3)
    F, _ = oracle.collapse_point(h6, correction=0)
    assert abs(F - delta / x3) < 1e-13 * delta
    # LPT overestimates the spherical collapse time: x3 > delta_c
    assert x3 > oracle.delta_c()


@pytest.mark.parametrize("delta", [0.05, 0.8, 1.686, 3.0, 10.0])
def test_sphere_corrected_gives_delta_over_delta_c(delta):
    g = _golden("spherical_collapse.txt")
    dc = float(g["delta_c_decimal"])
    assert abs(oracle.delta_c() - 3 / 20 * (12 * np.pi) ** (2 / 3)) < 1e-15
    assert abs(oracle.delta_c() - dc) < 1e-13
    rng = np.random.default_rng(4)
    Q = _random_rotation(rng)
    A = Q @ np.diag([delta / 3] * 3) @ Q.T  # a rotated sphere is still a sphere
    F, _ = oracle.collapse_point(_h6(A), correction=1)
    assert abs(F - delta / dc) < 1e-12 * delta


@pytest.mark.parametrize("delta", [-0.1, -2.0])
def test_underdense_sphere_never_collapses(delta):
    h6 = np.array([delta / 3] * 3 + [0.0] * 3)
    for corr in (0, 1):
        F, _ = oracle.collapse_point(h6, correction=corr)
        assert F == 0.0


@pytest.mark.parametrize("l1", [1e-4, 0.3, 1.0, 5.0])
def test_one_axis_is_zeldovich(l1):
    """lambda2 = lambda3 = 0: all higher orders vanish and the first axis
    collapses at D = 1/lambda1 (Zel'dovich), F = lambda1."""
    rng = np.random.default_rng(9)
    Q = _random_rotation(rng)
    A = Q @ np.diag([l1, 0.0, 0.0]) @ Q.T
    F, lam = oracle.collapse_point(_h6(A), correction=0)
    assert abs(F - l1) < 1e-12 * l1 + 1e-15
    F1, _ = oracle.collapse_point(_h6(A), correction=1)
    assert abs(F1 - l1) < 1e-12 * l1 + 1e-15


def test_second_order_trace_is_2lpt():
    """Sum over axes of the D^2 terms is (3/7) mu2 D^2: the divergence of the
    standard second-order LPT displacement.  Also: the split is covariant under
    permutation of the eigenvalues."""
    rng = np.random.default_rng(6)
    for _ in range(50):
        lam = rng.normal(size=3)
        mu2 = lam[0] * lam[1] + lam[0] * lam[2] + lam[1] * lam[2]
        c = np.array([oracle.axis_coeffs(lam, i) for i in range(3)])
        assert abs(c[:, 1].sum() - 3 / 7 * mu2) < 1e-13
        perm = rng.permutation(3)
        cp = np.array([oracle.axis_coeffs(lam[perm], i) for i in range(3)])
        assert np.allclose(cp, c[perm], rtol=0, atol=1e-14)


def _first_root_scan(c, npts=1_000_000):
    c1, c2, c3 = c
    p = lambda d: ((c3 * d + c2) * d + c1) * d - 1.0
    # scan a log grid wide enough to bracket any root of these magnitudes
    d = np.concatenate([[0.0], np.logspace(-6, 8, npts)])
    v = p(d)
    idx = np.nonzero(v >= 0)[0]
    if idx.size == 0:
        return np.inf
    i = idx[0]
    lo, hi = d[i - 1], d[i]
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if p(mid) < 0:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


def test_first_root_matches_brute_force_scan():
    rng = np.random.default_rng(8)
    for _ in range(300):
        c = rng.normal(size=3) * np.array([1.0, 0.7, 0.4])
        got = oracle.first_root(c)
        ref = _first_root_scan(c)
        if np.isinf(ref):
            # the scan reaches D = 1e8; the oracle's bound is exact
            assert np.isinf(got) or got > 1e7
        else:
            assert abs(got - ref) < 1e-9 * ref, (c, got, ref)


def test_first_root_degenerate_degrees():
    assert abs(oracle.first_root([2.0, 0.0, 0.0]) - 0.5) < 1e-15
    assert np.isinf(oracle.first_root([-1.0, 0.0, 0.0]))
    assert np.isinf(oracle.first_root([0.0, 0.0, 0.0]))
    # quadratic: c2 D^2 + c1 D - 1 = 0
    c1, c2 = 0.5, 0.25
    ref = (-c1 + np.sqrt(c1 ** 2 + 4 * c2)) / (2 * c2)
    assert abs(oracle.first_root([c1, c2, 0.0]) - ref) < 1e-14 * ref
    # tangent touch: p(D) = (1/3)(D - 1)^2 (D - 3) has a double root at D = 1,
    # where p reaches 0 at a local maximum; it is the first root.
    got = oracle.first_root([7 / 3, -5 / 3, 1 / 3])
    assert abs(got - 1.0) < 1e-6


# --------------------------------------------- collapse entry points pins --

def test_collapse_F_is_collapse_point_of_the_diagonal():
    """collapse_F takes sorted eigenvalues; on a diagonal Hessian (no rotation
    needed) it must equal collapse_point, whose pins above cover the model."""
    rng = np.random.default_rng(31)
    for _ in range(200):
        lam = np.sort(rng.normal(size=3))[::-1]
        for corr in (0, 1):
            F, l = oracle.collapse_point(_h6(np.diag(lam)), correction=corr)
            assert np.allclose(l, lam, rtol=0, atol=1e-15)
            assert abs(oracle.collapse_F(lam, corr) - F) <= 1e-14 * max(1.0, abs(F))
    # spheres: delta/x3 without the correction, delta/delta_c with it
    for delta in (0.3, 1.7, 4.0):
        lam = np.full(3, delta / 3)
        assert abs(oracle.collapse_F(lam, 0) - delta / oracle.x3()) < 1e-12
        assert abs(oracle.collapse_F(lam, 1) - delta / oracle.delta_c()) < 1e-12


def test_collapse_slope_closed_forms():
    """D a'(D) at the collapse root: 1 for one axis (a = D lambda1); for a
    sphere of linear contrast x at collapse, x/3 + 2x^2/21 + 69x^3/1701 at
    x = x3 (the derivative of the series that defines x3); 0 for a void."""
    for l1 in (0.5, 2.0, 7.0):
        assert abs(oracle.collapse_slope(np.array([l1, 0.0, 0.0])) - 1.0) < 1e-12
    x = oracle.x3()
    ref = x / 3 + 2 * x * x / 21 + 69 * x ** 3 / 1701
    for delta in (0.8, 2.5):
        assert abs(oracle.collapse_slope(np.full(3, delta / 3)) - ref) < 1e-10
    assert oracle.collapse_slope(np.array([-0.1, -0.2, -0.3])) == 0.0


def test_sampled_and_from_hessians_entry_points_equal_the_full_run():
    """The two partial entry points (sampled grid points; a stack of given
    Hessians) reproduce the full oracle run exactly at the same points: the
    same FP64 arithmetic, only the bookkeeping differs."""
    n, box = 16, 64.0
    d = _field(n, box, 32)
    radii = ic.log_radii(box / n, 16.0, 5)
    full = oracle.collapse_times(d, box, radii)
    q = np.random.default_rng(33).choice(n ** 3, size=300, replace=False)
    sam = oracle.collapse_times_sampled(d, box, radii, q)
    for k in ("fmax", "idx", "f2", "idx2"):
        assert np.array_equal(sam[k], full[k][q]), k
    hs = np.stack([oracle.hessian(d, box, R)[0].reshape(6, -1).T[q] for R in radii])
    fh = oracle.collapse_from_hessians(hs)
    for k in ("fmax", "idx"):
        assert np.array_equal(fh[k], full[k][q]), k
    # the runner-up and its index where a runner-up exists
    ok = full["idx2"][q] >= 0
    assert np.array_equal(fh["idx2"][ok], full["idx2"][q][ok])
    assert np.array_equal(fh["f2"][ok], full["f2"][q][ok])


# ------------------------------------------------------- running max pins --

def test_running_max_is_first_strict_argmax():
    n, box = 8, 50.0
    d = _field(n, box, 21)
    radii = ic.log_radii(box / n, 12.0, 6)
    out = oracle.collapse_times(d, box, radii, keep_all=True)
    fa = out["f_all"]
    ref_max = np.maximum(fa.max(axis=0), 0.0)
    assert np.array_equal(out["fmax"], ref_max)
    ref_idx = np.where(fa.max(axis=0) > 0, fa.argmax(axis=0), -1)
    assert np.array_equal(out["idx"], ref_idx)
    # the runner-up is the best of the other scales
    fa2 = fa.copy()
    fa2[out["idx"][out["idx"] >= 0], np.nonzero(out["idx"] >= 0)[0]] = -np.inf
    ok = out["idx"] >= 0
    assert np.allclose(out["f2"][ok], np.maximum(fa2.max(axis=0)[ok], 0.0))


def test_pipeline_agrees_with_pointwise_composition():
    n, box = 8, 50.0
    d = _field(n, box, 5)
    radii = ic.log_radii(box / n, 12.0, 4)
    out = oracle.collapse_times(d, box, radii, keep_all=True)
    for s, r in enumerate(radii):
        h, _ = oracle.hessian(d, box, r)
        flat = h.reshape(6, -1)
        for q in (0, 17, 200, 511):
            F, _ = oracle.collapse_point(flat[:, q], correction=1)
            assert F == out["f_all"][s, q]


# ------------------------------------------------------ displacement pins --

@pytest.mark.parametrize("mode", [(1, 2, 3), (5, 1, 2), (0, 0, 2), (4, 0, 1)])
def test_displacement_single_mode_closed_form(mode):
    """psi = i k delta / k^2 for one mode gives
    psi(q) = -(k / k^2) 2 Im(A e^{i k.q}) / n^3 (zero along a Nyquist axis)."""
    n, box = 8, 40.0
    d = np.zeros((n, n, n // 2 + 1), dtype=np.complex128)
    amp = 0.4 + 0.9j
    mx, my, mz = mode
    d[mx, my, mz] = amp
    if mz == 0:
        d[(-mx) % n, (-my) % n, 0] = np.conj(amp)
    psi = oracle.displacement(d, box)
    s = [mx if mx < n // 2 else mx - n, my if my < n // 2 else my - n, mz]
    kf = 2 * np.pi / box
    k = kf * np.array(s, dtype=float)
    k2 = k @ k
    q = np.indices((n, n, n))
    phase = 2 * np.pi * (s[0] * q[0] + s[1] * q[1] + s[2] * q[2]) / n
    wave = -2 * np.imag(amp * np.exp(1j * phase)) / n ** 3
    for c in range(3):
        ref = np.zeros_like(wave) if s[c] == -n // 2 else k[c] / k2 * wave
        assert np.abs(psi[c] - ref).max() < 1e-15 + 1e-12 * np.abs(wave).max()


def test_displacement_divergence_is_minus_delta():
    """-div psi = delta, checked in real space with numpy's spectral derivative
    (a library routine), away from the odd-order Nyquist modes."""
    n, box = 12, 60.0
    d = _field(n, box, 9)
    # drop every mode with a Nyquist index so the spectral derivative is exact
    d[n // 2, :, :] = 0
    d[:, n // 2, :] = 0
    d[:, :, n // 2] = 0
    psi = oracle.displacement(d, box)
    kf = 2 * np.pi / box
    div = 0
    for c in range(3):
        f = np.fft.rfftn(psi[c], axes=(0, 1, 2))
        m = np.fft.fftfreq(n, 1.0 / n) if c < 2 else np.arange(n // 2 + 1)
        shape = [1, 1, 1]
        shape[c] = -1
        div = div + np.fft.irfftn(1j * kf * m.reshape(shape) * f, s=(n, n, n), axes=(0, 1, 2))
    ref = np.fft.irfftn(d, s=(n, n, n), axes=(0, 1, 2))
    assert np.abs(-div - ref).max() < 1e-11 * np.abs(ref).max()


def test_multi_point_direct_sum_matches_fft_path():
    n, box, radius = 16, 90.0, 4.0
    d = _field(n, box, 13)
    h, _ = oracle.hessian(d, box, radius)
    rng = np.random.default_rng(1)
    q = rng.integers(0, n ** 3, size=7)
    got = oracle.hessian_points(d, box, radius, q)
    ref = h.reshape(6, -1)[:, q].T
    assert np.abs(got - ref).max() < 1e-12 * np.abs(h).max()


@pytest.mark.parametrize("radius", [0.0, 3.0])
def test_smoothed_displacement_single_mode(radius):
    """psi_R = i k W(kR) delta / k^2: one mode gives the unsmoothed closed form
    times exp(-k^2 R^2 / 2)."""
    n, box = 8, 40.0
    d = np.zeros((n, n, n // 2 + 1), dtype=np.complex128)
    amp = 0.4 + 0.9j
    d[1, 2, 3] = amp
    psi = oracle.displacement(d, box, radius)
    s = [1, 2, 3]
    kf = 2 * np.pi / box
    k = kf * np.array(s, dtype=float)
    k2 = k @ k
    q = np.indices((n, n, n))
    phase = 2 * np.pi * (s[0] * q[0] + s[1] * q[1] + s[2] * q[2]) / n
    wave = -2 * np.imag(amp * np.exp(1j * phase)) / n ** 3 * np.exp(-0.5 * k2 * radius ** 2)
    for c in range(3):
        assert np.abs(psi[c] - k[c] / k2 * wave).max() < 1e-15 + 1e-12 * np.abs(wave).max()


@pytest.mark.parametrize("shape", [(8, 8, 8), (8, 12, 6)])
def test_vmax_is_displacement_at_the_argmax_radius(shape):
    box = 50.0
    if shape[0] == shape[1] == shape[2]:
        d = _field(shape[0], box, 23)
    else:
        d = _half_spectrum(np.random.default_rng(23).normal(size=shape))
    radii = ic.log_radii(box / shape[0], 12.0, 4)
    out = oracle.collapse_times(d, box, radii, velocities=True)
    v = out["vmax"].reshape(3, -1)
    n3 = int(np.prod(shape))
    checked = 0
    for q in (0, 100, 300, n3 - 1, n3 // 3):
        s = out["idx"][q]
        if s < 0:
            assert np.all(v[:, q] == 0)
        else:
            ref = oracle.displacement(d, box, radii[s]).reshape(3, -1)[:, q]
            assert np.allclose(v[:, q], ref, rtol=0, atol=1e-15)
            checked += 1
    assert checked > 0


# ---- fragmentation front end (Sec. 2.1.2): order and neighbours before ----

def _brute_fragment(F):
    """Straight from the definitions: sort the (F, q) pairs by a key, and
    count for each particle the neighbours whose pair comes first by direct
    comparison (larger F, or equal F and smaller index)."""
    nx, ny, nz = F.shape
    flat = [float(v) for v in F.ravel()]
    order = sorted(range(nx * ny * nz), key=lambda q: (-flat[q], q))
    nb = np.zeros((nx, ny, nz), dtype=np.int64)
    for x in range(nx):
        for y in range(ny):
            for z in range(nz):
                q = (x * ny + y) * nz + z
                for dx, dy, dz in ((1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)):
                    r = (((x + dx) % nx) * ny + (y + dy) % ny) * nz + (z + dz) % nz
                    if flat[r] > flat[q] or (flat[r] == flat[q] and r < q):
                        nb[x, y, z] += 1
    return np.array(order), nb


@pytest.mark.parametrize("shape,levels", [((3, 3, 3), 0), ((4, 4, 4), 5), ((5, 5, 5), 3), ((6, 6, 6), 0),
                                          ((3, 5, 4), 4), ((6, 2, 3), 0), ((2, 4, 7), 2)])
def test_fragment_order_brute_force(shape, levels):
    rng = np.random.default_rng(40 + sum(shape))
    F = rng.random(shape).astype(np.float32)
    if levels:  # many exact ties, including zeros (particles that never collapse)
        F = np.floor(F * levels).astype(np.float32) / levels
    order, nb = oracle.fragment_order(F)
    border, bnb = _brute_fragment(F)
    assert np.array_equal(order, border)
    assert np.array_equal(nb, bnb)


def test_fragment_order_invariants():
    rng = np.random.default_rng(7)
    n = 8
    F = np.maximum(rng.normal(size=(n, n, n)), 0).astype(np.float32)  # about half never collapse
    order, nb = oracle.fragment_order(F)
    assert np.array_equal(np.sort(order), np.arange(n ** 3))  # a permutation
    f = F.ravel()[order]
    assert np.all(np.diff(f) <= 0)  # descending F
    ties = np.nonzero(np.diff(f) == 0)[0]
    assert np.all(order[ties] < order[ties + 1])  # equal F: ascending index
    # each of the 3 n^3 neighbour pairs is counted by exactly one of its two ends
    assert nb.sum() == 3 * n ** 3
    assert nb.ravel()[order[0]] == 0 and nb.ravel()[order[-1]] == 6
    # all-equal field: the order is the index order, and q counts its smaller-index neighbours
    o2, nb2 = oracle.fragment_order(np.zeros((4, 4, 4), dtype=np.float32))
    assert np.array_equal(o2, np.arange(64))
    assert nb2[0, 0, 0] == 0 and nb2[3, 3, 3] == 6 and nb2[1, 1, 1] == 3


# ---- second-order LPT displacement ----

def _half_spectrum(field):
    """Forward-convention half-spectrum D(k) = sum_q d(q) e^{-ik.q} of a real
    field, in the [kx][ky][kz <= N/2] layout (numpy's rfftn)."""
    return np.fft.rfftn(field)


def test_2lpt_vanishes_for_a_plane_wave():
    # one Fourier mode: the deformation tensor has rank one, its second
    # invariant is zero, and the motion is exactly Zel'dovich
    n, box = 16, 64.0
    x = np.arange(n) * box / n
    X, Y, Z = np.meshgrid(x, x, x, indexing="ij")
    k = 2 * np.pi / box
    d = 0.7 * np.cos(2 * k * X + 3 * k * Y - k * Z)
    psi2 = oracle.displacement_2lpt(_half_spectrum(d), box)
    assert np.abs(psi2).max() < 1e-12


def test_2lpt_two_crossed_waves_closed_form():
    # delta = A cos(k1 x) + B cos(k2 y): phi_xx = A cos(k1 x), phi_yy = B cos(k2 y),
    # S = A B cos(k1 x) cos(k2 y) = (AB/2) [cos(K+.q) + cos(K-.q)], K+- = (k1, +-k2, 0),
    # and each c cos(K.q) gives psi2 = -(3/7) c K sin(K.q) / K^2
    n, box = 16, 64.0
    x = np.arange(n) * box / n
    X, Y, Z = np.meshgrid(x, x, x, indexing="ij")
    k1, k2 = 2 * np.pi * 2 / box, 2 * np.pi * 3 / box
    A, B = 0.8, -0.5
    d = A * np.cos(k1 * X) + B * np.cos(k2 * Y)
    psi2 = oracle.displacement_2lpt(_half_spectrum(d), box)
    K2 = k1 ** 2 + k2 ** 2
    sp, sm = np.sin(k1 * X + k2 * Y), np.sin(k1 * X - k2 * Y)
    c = -(3.0 / 7.0) * A * B / 2 / K2
    assert np.allclose(psi2[0], c * k1 * (sp + sm), atol=1e-12)
    assert np.allclose(psi2[1], c * k2 * (sp - sm), atol=1e-12)
    assert np.abs(psi2[2]).max() < 1e-12
    # div psi2 = -(3/7) S, read back spectrally from the result
    kk = 2 * np.pi * np.fft.fftfreq(n, d=box / n)
    div = sum(np.real(np.fft.ifftn(1j * np.meshgrid(kk, kk, kk, indexing="ij")[i] * np.fft.fftn(psi2[i])))
              for i in range(3))
    assert np.allclose(div, -(3.0 / 7.0) * A * B * np.cos(k1 * X) * np.cos(k2 * Y), atol=1e-12)


@pytest.mark.parametrize("shape", [(16, 8, 12), (12, 16, 8)])
def test_2lpt_two_crossed_waves_non_cubic(shape):
    """The crossed-wave closed form off the cube (cubic cells: the side along
    an axis of m points is box m / nx), waves along x and z: pins the per-axis
    wavenumbers of the second-order source and of its displacement."""
    nx, ny, nz = shape
    box = 48.0
    cell = box / nx
    X, Y, Z = np.meshgrid(np.arange(nx) * cell, np.arange(ny) * cell, np.arange(nz) * cell, indexing="ij")
    k1, k3 = 2 * np.pi * 2 / box, 2 * np.pi * 1 / (box * nz / nx)
    A, B = 0.6, 0.9
    d = A * np.cos(k1 * X) + B * np.cos(k3 * Z)
    psi2 = oracle.displacement_2lpt(_half_spectrum(d), box)
    K2 = k1 ** 2 + k3 ** 2
    sp, sm = np.sin(k1 * X + k3 * Z), np.sin(k1 * X - k3 * Z)
    c = -(3.0 / 7.0) * A * B / 2 / K2
    assert np.allclose(psi2[0], c * k1 * (sp + sm), atol=1e-12)
    assert np.abs(psi2[1]).max() < 1e-12
    assert np.allclose(psi2[2], c * k3 * (sp - sm), atol=1e-12)


# ---- non-cubic grids (cubic cells: the side along an axis of m points is box m / nx) ----

@pytest.mark.parametrize("shape,mode", [((8, 12, 16), (1, 2, 3)), ((16, 8, 12), (5, 1, 2)), ((12, 16, 8), (0, 7, 1)),
                                        ((8, 16, 12), (3, 0, 0))])
def test_single_mode_closed_form_non_cubic(shape, mode):
    """A single mode on an nx x ny x nz grid: phi_ij(q) = (k_i k_j / k^2) W(k)
    2 Re(A e^{i k.q}) / (nx ny nz) with k_i = 2 pi s_i / L_i and
    k.q = 2 pi sum_i s_i q_i / n_i: pins the per-axis wavenumbers, the axis
    order and the normalisation off the cube."""
    nx, ny, nz = shape
    box, radius = 40.0, 2.0
    L = np.array([box, box * ny / nx, box * nz / nx])
    d = np.zeros((nx, ny, nz // 2 + 1), dtype=np.complex128)
    amp = 0.4 + 0.9j
    mx, my, mz = mode
    d[mx, my, mz] = amp
    if mz == 0:
        d[(-mx) % nx, (-my) % ny, 0] = np.conj(amp)
    h, _ = oracle.hessian(d, box, radius)
    s = np.array([mx if mx < nx // 2 else mx - nx, my if my < ny // 2 else my - ny, mz])
    k = 2 * np.pi * s / L
    k2 = k @ k
    q = np.indices(shape)
    phase = 2 * np.pi * (s[0] * q[0] / nx + s[1] * q[1] / ny + s[2] * q[2] / nz)
    wave = 2 * np.real(amp * np.exp(1j * phase)) / (nx * ny * nz)
    w = np.exp(-0.5 * k2 * radius ** 2)
    for c, (i, j) in enumerate([(0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2)]):
        ref = k[i] * k[j] / k2 * w * wave
        assert np.abs(h[c] - ref).max() < 1e-14 + 1e-12 * np.abs(wave).max(), (c, shape, mode)


@pytest.mark.parametrize("shape,radius", [((8, 16, 12), 3.0), ((16, 12, 8), 0.0)])
def test_trace_and_displacement_divergence_non_cubic(shape, radius):
    """Off the cube: the trace of the Hessian is the smoothed delta and the
    divergence of the displacement is minus delta, both against numpy's irfftn
    of a random Hermitian spectrum (numpy's rfftn of a real field)."""
    nx, ny, nz = shape
    box = 48.0
    L = [box, box * ny / nx, box * nz / nx]
    d = np.fft.rfftn(np.random.default_rng(5).normal(size=shape))
    d[0, 0, 0] = 0.0
    kx = 2 * np.pi * np.fft.fftfreq(nx, 1.0 / nx) / L[0]
    ky = 2 * np.pi * np.fft.fftfreq(ny, 1.0 / ny) / L[1]
    kz = 2 * np.pi * np.arange(nz // 2 + 1) / L[2]
    k2 = kx[:, None, None] ** 2 + ky[None, :, None] ** 2 + kz[None, None, :] ** 2
    h, _ = oracle.hessian(d, box, radius)
    ref = np.fft.irfftn(d * np.exp(-0.5 * k2 * radius ** 2), s=shape, axes=(0, 1, 2))
    assert np.abs(h[0] + h[1] + h[2] - ref).max() < 1e-12 * np.abs(ref).max()
    psi = oracle.displacement(d, box, 0.0)
    # divergence spectrally, Nyquist components of each derivative dropped as in psi
    kxs, kys = kx.copy(), ky.copy()
    kxs[nx // 2] = 0.0
    kys[ny // 2] = 0.0
    kzs = kz.copy()
    kzs[-1] = 0.0
    kk = [kxs[:, None, None], kys[None, :, None], kzs[None, None, :]]
    div = sum(np.fft.irfftn(1j * kk[i] * np.fft.rfftn(psi[i]), s=shape, axes=(0, 1, 2)) for i in range(3))
    lapl = np.fft.irfftn(-d * (kk[0] ** 2 + kk[1] ** 2 + kk[2] ** 2) / np.where(k2 > 0, k2, 1.0), s=shape,
                         axes=(0, 1, 2))
    assert np.abs(div - lapl).max() < 1e-11 * np.abs(lapl).max()


# ---- variance of the field after smoothing (radius schedule) ----

@pytest.mark.parametrize("shape,radius", [((8, 8, 8), 0.0), ((8, 12, 16), 3.0), ((16, 8, 12), 7.5)])
def test_sigma2_flat_spectrum_closed_form(shape, radius):
    """With a flat spectrum P = A the sum separates:
    sigma^2 = (A / V) (prod_i theta_i - 1), theta_i = sum_m exp(-(2 pi m / L_i)^2 R^2)."""
    A, box = 2.5, 30.0
    nx, ny, nz = shape
    L = [box, box * ny / nx, box * nz / nx]
    theta = [np.sum(np.exp(-(2 * np.pi * (np.arange(n) - n // 2) / Li) ** 2 * radius ** 2))
             for n, Li in zip(shape, L)]
    ref = A / (L[0] * L[1] * L[2]) * (theta[0] * theta[1] * theta[2] - 1.0)
    got = oracle.sigma2(shape, box, radius, power=lambda k: np.full(k.shape, A))
    assert abs(got - ref) <= 1e-13 * ref


# ------------------------------------------------- conditioning interval --

def _rotated(lam, seed):
    """h6 of R diag(lam) R^T for a random rotation R."""
    rng = np.random.default_rng(seed)
    q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
    a = q @ np.diag(lam) @ q.T
    return np.array([a[0, 0], a[1, 1], a[2, 2], a[0, 1], a[0, 2], a[1, 2]])


def test_collapse_interval_zero_width_is_collapse_F():
    rng = np.random.default_rng(7)
    lams = np.sort(rng.normal(scale=0.8, size=(20, 3)), axis=1)[:, ::-1]
    h = np.stack([_rotated(l, i) for i, l in enumerate(lams)])[None]
    for corr in (0, 1):
        lo, hi = oracle.collapse_interval(h, [0.5], 0.0, corr)
        ref = np.array([oracle.collapse_F(l, corr) for l in lams])
        assert np.allclose(lo[0], ref, rtol=1e-12, atol=1e-13)
        assert np.allclose(hi[0], ref, rtol=1e-12, atol=1e-13)


@pytest.mark.parametrize("a", [0.3, 0.7, 1.2])
def test_collapse_interval_contains_the_perturbed_spheres(a):
    """A sphere lambda = (a, a, a) with half-width d = u (hscale + a): the
    corners (a +- d)(1, 1, 1) are spheres, F = 3 (a +- d) / delta_c exactly
    (corrected mode), so the interval must reach both."""
    u, hs = 1e-3, 0.2
    d = u * (hs + a)
    lo, hi = oracle.collapse_interval(np.array([[[a, a, a, 0.0, 0.0, 0.0]]]), [hs], u, 1)
    dc = oracle.delta_c()
    assert hi[0, 0] >= 3 * (a + d) / dc - 1e-12
    assert lo[0, 0] <= 3 * (a - d) / dc + 1e-12
    # smooth there: the interval stays of the order of d |grad F|
    assert hi[0, 0] - lo[0, 0] < 20 * d


def _tangent_lambda1(l2, l3):
    """lambda1 at which the axis-0 displacement a(D) has a local maximum equal
    to 1 (a tangent first crossing), by bisection on the maximum's value; the
    coefficients come from the oracle and the maximum from numpy's roots."""
    def peak(t):
        c1, c2, c3 = oracle.axis_coeffs(np.array([t, l2, l3]), 0)
        r = np.roots([3 * c3, 2 * c2, c1])
        r = np.sort(r[np.isreal(r)].real)
        r = r[r > 0]
        return (c1 * r[0] + c2 * r[0] ** 2 + c3 * r[0] ** 3) if r.size else np.inf
    lo, hi = l2, 0.32
    assert peak(lo) < 1 < peak(hi)
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if peak(mid) < 1:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


def test_collapse_interval_spans_a_tangent_jump():
    """At a tangent first crossing F jumps: just above the tangent eigenvalue
    the axis collapses at the tangent point, just below only much later.  A
    tiny half-width must give an interval as wide as that jump; the same
    half-width away from the tangency gives an interval of width ~d."""
    l2, l3 = 0.2, -0.5
    t = _tangent_lambda1(l2, l3)
    above = oracle.collapse_F(np.array([t * (1 + 1e-7), l2, l3]), 0)
    below = oracle.collapse_F(np.array([t * (1 - 1e-7), l2, l3]), 0)
    jump = above - below
    assert jump > 0.05 * above  # the jump is real
    u = 1e-6
    lo, hi = oracle.collapse_interval(np.array([[[t, l2, l3, 0, 0, 0]]]), [0.0], u, 0)
    assert hi[0, 0] - lo[0, 0] >= 0.9 * jump
    lo2, hi2 = oracle.collapse_interval(np.array([[[0.8 * t, l2, l3, 0, 0, 0]]]), [0.0], u, 0)
    assert hi2[0, 0] - lo2[0, 0] < 1e-3 * jump
