"""The CUDA path's per-particle arithmetic (csrc/collapse.cuh, compiled for
the host) against the FP64 oracle: eigenvalues and collapse time F in FP64
and FP32 on random triplets and on the limits (sphere, one axis)."""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
OUT = os.path.join(ROOT, "paper_1305_1505_gb300", "_build", "libcollapse_host.so")
DP = ctypes.POINTER(ctypes.c_double)


@pytest.fixture(scope="module")
def lib():
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    os.makedirs(os.path.dirname(OUT), exist_ok=True)
    subprocess.check_call([nvcc, "-O2", "-std=c++17", "-shared", "-Xcompiler", "-fPIC",
                           "-I", os.path.join(ROOT, "paper_1305_1505_gb300", "csrc"),
                           "-o", OUT, os.path.join(HERE, "collapse_host.cu")])
    L = ctypes.CDLL(OUT)
    L.host_collapse.argtypes = [DP, ctypes.c_int, ctypes.c_int, ctypes.c_double, DP]
    L.host_collapse.restype = ctypes.c_double
    L.host_eig.argtypes = [DP, DP, ctypes.c_int]
    L.host_eig.restype = ctypes.c_double
    L.host_bound.argtypes = [DP, ctypes.c_int, ctypes.c_int, ctypes.c_double]
    L.host_bound.restype = ctypes.c_double
    return L


def _F(L, lam, corr, use_float):
    lam = np.ascontiguousarray(lam, dtype=np.float64)
    k = ctypes.c_double()
    dcorr = 1 / oracle.delta_c() - 1 / oracle.x3()
    return L.host_collapse(lam.ctypes.data_as(DP), corr, use_float, dcorr, ctypes.byref(k)), k.value


def test_collapse_fp64_matches_oracle(lib):
    rng = np.random.default_rng(0)
    for _ in range(5000):
        lam = np.sort(rng.normal(size=3) * 0.6)[::-1]
        for corr in (0, 1):
            g, _ = _F(lib, lam, corr, 0)
            o = oracle.collapse_F(lam, corr)
            assert abs(g - o) <= 1e-10 * max(1.0, abs(o)), (lam, corr, g, o)


def test_collapse_fp32_within_tolerance_or_flagged(lib):
    rng = np.random.default_rng(1)
    for _ in range(5000):
        lam = np.sort(rng.normal(size=3) * 0.6)[::-1]
        g, kap = _F(lib, lam, 1, 1)
        o = oracle.collapse_F(lam, 1)
        if kap >= 1e-3:  # not sent to the FP64 redo
            assert abs(g - o) <= 1e-4 * abs(o) + 1e-6, (lam, g, o, kap)


@pytest.mark.parametrize("delta", [0.1, 1.0, 4.0])
def test_limits(lib, delta):
    g, _ = _F(lib, [delta / 3] * 3, 1, 0)
    assert abs(g - delta / oracle.delta_c()) < 1e-12 * delta
    g, _ = _F(lib, [delta, 0.0, 0.0], 0, 0)
    assert abs(g - delta) < 1e-12 * delta
    g, _ = _F(lib, [-delta / 3] * 3, 1, 0)
    assert g == 0.0


def test_eigen_fp64_and_fp32(lib):
    rng = np.random.default_rng(2)
    for _ in range(3000):
        h = rng.normal(size=6)
        for use_float, tol in ((0, 1e-12), (1, 2e-5)):
            lam = np.empty(3)
            r = lib.host_eig(h.ctypes.data_as(DP), lam.ctypes.data_as(DP), use_float)
            ref = oracle.eig3(h)
            if use_float and 1 - r < 2e-4:
                continue  # near-degenerate: the kernel redoes these in FP64
            assert np.abs(lam - ref).max() <= tol * np.abs(h).max(), (h, lam, ref)


def _structured(rng):
    """Spheres, one- and two-axis triples, zeros, sign mixes, exact ties, a
    root crossing zero (lam0 -> 0+ with the others negative), and random
    triples over six decades of amplitude."""
    rows = []
    for t in (-2.0, -0.3, 0.0, 1e-4, 0.2, 1.0, 3.0):
        rows += [(t, t, t), (t, 0.0, 0.0), (t, t, 0.0), (t, 0.0, -t), (t, -t, -t), (0.0, 0.0, t)]
    for eps in (1e-7, 1e-6, 1e-5, 1e-4, 1e-3):
        for a, b in rng.uniform(0.01, 0.4, size=(40, 2)):
            rows.append((eps, -min(a, b), -max(a, b)))
    for amp in (1e-3, 1e-2, 0.1, 1.0, 10.0, 100.0):
        rows += [tuple(r) for r in rng.normal(size=(300, 3)) * amp]
        rows += [(u, u, v) for u, v in rng.normal(size=(60, 2)) * amp]
        rows += [(u, v, v) for u, v in rng.normal(size=(60, 2)) * amp]
    return -np.sort(-np.array(rows, dtype=np.float64), axis=1)


def test_collapse_fp32_structured(lib):
    lam_all = _structured(np.random.default_rng(12))
    flagged = 0
    for lam in lam_all:
        g, kap = _F(lib, lam, 1, 1)
        o = oracle.collapse_F(lam, 1)
        scale = np.abs(lam).max()
        assert np.isfinite(kap), (lam, g, kap)
        if kap >= 1e-3:
            assert np.isfinite(g) and abs(g - o) <= 1e-4 * abs(o) + 1e-6 * scale, (lam, g, o, kap)
        else:
            assert np.isfinite(g), (lam, g, kap)
            flagged += 1
        if o == 0.0 and kap >= 1e-3:
            assert g == 0.0, (lam, g)
    assert flagged <= 0.02 * len(lam_all)


def test_fp32_eigenvalue_absolute_error_bound(lib):
    """The FP32 trigonometric eigenvalues are accurate to ~1e-6 of the matrix
    scale in absolute terms, not relative to each eigenvalue: a largest
    eigenvalue far below the scale (a direction the smoothing has emptied,
    which the method's radii never produce systematically) keeps only that
    absolute accuracy.  This pins the bound the design relies on."""
    rng = np.random.default_rng(21)
    worst = 0.0
    for t in range(2000):
        lam = -np.sort(-rng.normal(size=3) * 10 ** rng.uniform(-3, 1))
        Q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
        A = Q @ np.diag(lam) @ Q.T
        h = np.array([A[0, 0], A[1, 1], A[2, 2], A[0, 1], A[0, 2], A[1, 2]])
        h32 = h.astype(np.float32).astype(np.float64)
        ref = np.sort(oracle.eig3(h32))[::-1]
        got = np.empty(3)
        r = lib.host_eig(np.ascontiguousarray(h32).ctypes.data_as(DP), got.ctypes.data_as(DP), 1)
        if r > 1 - 2e-4:
            continue  # near-degenerate: redone in FP64
        worst = max(worst, np.abs(got - ref).max() / np.abs(ref).max())
    assert worst < 4e-6, worst


def _rotated(lam, rng):
    """h = R diag(lam) R^T for a random rotation R, as (xx, yy, zz, xy, xz, yz)."""
    R, _ = np.linalg.qr(rng.normal(size=(3, 3)))
    A = R @ np.diag(lam) @ R.T
    return np.array([A[0, 0], A[1, 1], A[2, 2], A[0, 1], A[0, 2], A[1, 2]])


def test_invariant_bound_above_F(lib):
    """collapse_bound (which clears FP64-redo candidates that cannot beat
    their running maximum) is an upper bound on F: over spheres, one- and
    two-axis triples, ties, sign mixes and six decades of amplitude, in random
    orientations, the oracle's F never exceeds it (FP64 bound, and the FP32
    bound within its rounding)."""
    k = 1.54
    assert k ** 3 - k ** 2 - 3 / 7 * k - (40 / 84 + 1 / 9) > 0.03  # the root bound's margin
    dcorr = 1 / oracle.delta_c() - 1 / oracle.x3()
    assert dcorr > 0
    rng = np.random.default_rng(13)
    worst = 0.0
    for lam in _structured(rng):
        h = _rotated(lam, rng)
        hc = np.ascontiguousarray(h)
        scale = np.abs(lam).max()
        for corr in (0, 1):
            F, _ = oracle.collapse_point(h, corr)
            b64 = lib.host_bound(hc.ctypes.data_as(DP), corr, 0, dcorr)
            b32 = lib.host_bound(hc.ctypes.data_as(DP), corr, 1, dcorr)
            assert F <= b64 * (1 + 1e-12), (lam, corr, F, b64)
            assert F <= b32 * (1 + 1e-6) + 1e-7 * scale, (lam, corr, F, b32)
            if b64 > 0:
                worst = max(worst, F / b64)
        # the diagonal form (the redo's entries that carry eigenvalues)
        d = np.ascontiguousarray([lam[0], lam[1], lam[2], 0.0, 0.0, 0.0])
        F, _ = oracle.collapse_point(d, 1)
        assert F <= lib.host_bound(d.ctypes.data_as(DP), 1, 0, dcorr) * (1 + 1e-12)
    print("largest F / bound: %.3f" % worst)
    assert worst < 1.0
    z = np.zeros(6)
    assert lib.host_bound(z.ctypes.data_as(DP), 1, 0, dcorr) == 0.0


def test_fp32_gap_for_small_largest_eigenvalue(lib):
    """The documented FP32 accuracy gap: when the largest eigenvalue is a
    small fraction eps of the matrix scale (a direction the smoothing has
    emptied), the FP32 eigenvalues' absolute error (~1e-7 of the scale, pinned
    above) becomes a relative error of F that grows like 1/eps.  Measured on
    the host build of the CUDA path's FP32 eigenvalues and collapse from FP32
    Hessians, against the oracle: within the 1e-4 parity tolerance down to
    eps = 1e-3, beyond it below 1e-4, and bounded by 1e-7 / eps throughout."""
    dcorr = 1 / oracle.delta_c() - 1 / oracle.x3()
    rng = np.random.default_rng(5)
    worst = {}
    for eps in (1e-2, 1e-3, 1e-4, 1e-5):
        w = 0.0
        for _ in range(300):
            a, b = rng.uniform(0.2, 1.0, 2)
            lam = -np.sort(-np.array([eps, -a, -b]))
            h = _rotated(lam, rng).astype(np.float32).astype(np.float64)
            l32 = np.empty(3)
            r = lib.host_eig(np.ascontiguousarray(h).ctypes.data_as(DP), l32.ctypes.data_as(DP), 1)
            if r > 1 - 2e-4:
                continue  # near-degenerate: redone in FP64
            k = ctypes.c_double()
            F32 = lib.host_collapse(np.ascontiguousarray(l32).ctypes.data_as(DP), 1, 1, dcorr, ctypes.byref(k))
            F = oracle.collapse_F(np.sort(oracle.eig3(h))[::-1], 1)
            if F > 0 and k.value >= 1e-3:
                w = max(w, abs(F32 - F) / F)
        worst[eps] = w
        assert w <= 1e-7 / eps, (eps, w)
    print("worst relative F error by eps:", worst)
    assert worst[1e-3] < 1e-4 and worst[1e-5] > 1e-4
