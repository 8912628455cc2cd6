"""The per-particle eigenvalue and collapse arithmetic compiled for sm_103a
and run on the GPU, one particle per thread, against the FP64 oracle."""
import ctypes
import os
import subprocess

import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
OUT = os.path.join(ROOT, "paper_1305_1505_gb300", "_build", "libcollapse_device.so")
DP = ctypes.POINTER(ctypes.c_double)


@pytest.fixture(scope="module")
def lib():
    os.makedirs(os.path.dirname(OUT), exist_ok=True)
    subprocess.check_call(["/usr/local/cuda/bin/nvcc", "-gencode", "arch=compute_103a,code=sm_103a",
                           "-O3", "-std=c++17", "-shared", "-Xcompiler", "-fPIC",
                           "-Werror", "cross-execution-space-call",
                           "-I", os.path.join(ROOT, "paper_1305_1505_gb300", "csrc"),
                           "-o", OUT, os.path.join(HERE, "collapse_device.cu")])
    L = ctypes.CDLL(OUT)
    L.dev_eval.argtypes = [DP, DP, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_int,
                           DP, DP, DP]
    L.dev_eval.restype = ctypes.c_int
    return L


def _eval(L, lam, h, corr, use_float):
    if use_float == 2 and lam.shape[0] % 2:  # pairs need an even count
        lam, h = np.vstack([lam, lam[:1]]), np.vstack([h, h[:1]])
        F, kap, eig = _eval(L, lam, h, corr, use_float)
        return F[:-1], kap[:-1], eig[:-1]
    n = lam.shape[0]
    lam = np.ascontiguousarray(lam, dtype=np.float64)
    h = np.ascontiguousarray(h, dtype=np.float64)
    F, kap, eig = np.empty(n), np.empty(n), np.empty((n, 3))
    dcorr = 1 / oracle.delta_c() - 1 / oracle.x3()
    assert L.dev_eval(lam.ctypes.data_as(DP), h.ctypes.data_as(DP), n, corr, dcorr, use_float,
                      F.ctypes.data_as(DP), kap.ctypes.data_as(DP), eig.ctypes.data_as(DP)) == 0
    return F, kap, eig


@pytest.mark.parametrize("mode", [1, 2], ids=["fp32", "fp32_pairs"])
def test_device_collapse_and_eigen_vs_oracle(lib, mode):
    rng = np.random.default_rng(3)
    n = 20000
    lam = -np.sort(-rng.normal(size=(n, 3)) * 0.6, axis=1)
    h = rng.normal(size=(n, 6))
    ref = np.array([oracle.collapse_F(l, 1) for l in lam])
    ref_eig = np.array([oracle.eig3(x) for x in h])
    F64, _, e64 = _eval(lib, lam, h, 1, 0)
    assert np.abs(F64 - ref).max() <= 1e-10 * max(1.0, np.abs(ref).max())
    assert np.abs(e64 - ref_eig).max() <= 1e-12 * np.abs(h).max()
    F32, kap, e32 = _eval(lib, lam, h, 1, mode)
    ok = kap >= 1e-3
    err = np.abs(F32 - ref)
    bad = np.nonzero(ok & (err > 1e-4 * np.abs(ref) + 1e-6))[0]
    assert bad.size == 0, (bad[:5], lam[bad[:5]], F32[bad[:5]], ref[bad[:5]])
    hmax = np.abs(h).max(axis=1)
    eerr = np.abs(e32 - ref_eig).max(axis=1) / hmax
    assert np.percentile(eerr, 99.9) < 1e-5


def _special_eigenvalues(rng):
    """Structured and scaled eigenvalue triples (sorted, largest first):
    spheres, one- and two-axis cases, zero and sign-mixed triples, exact
    diagonal ties, roots crossing zero (lam0 -> 0+ with the others negative),
    and random triples over six decades of amplitude."""
    rows = []
    for t in (-2.0, -0.3, 0.0, 1e-4, 0.2, 1.0, 3.0):
        rows += [(t, t, t), (t, 0.0, 0.0), (t, t, 0.0), (t, 0.0, -t), (t, -t, -t), (0.0, 0.0, t)]
    for eps in (1e-7, 1e-6, 1e-5, 1e-4, 1e-3):
        for a, b in rng.uniform(0.01, 0.4, size=(200, 2)):
            rows.append((eps, -min(a, b), -max(a, b)))
    for amp in (1e-3, 1e-2, 0.1, 1.0, 10.0, 100.0):
        x = rng.normal(size=(2000, 3)) * amp
        rows += [tuple(r) for r in x]
        a = rng.normal(size=(500, 2)) * amp
        rows += [(u, u, v) for u, v in a] + [(u, v, v) for u, v in a]
    lam = -np.sort(-np.array(rows, dtype=np.float64), axis=1)
    return lam


@pytest.mark.parametrize("mode", [1, 2], ids=["fp32", "fp32_pairs"])
def test_device_collapse_special_cases(lib, mode):
    lam = _special_eigenvalues(np.random.default_rng(11))
    h = np.zeros((lam.shape[0], 6))
    h[:, :3] = lam
    ref = np.array([oracle.collapse_F(l, c) for l in lam for c in (1,)])
    F32, kap, _ = _eval(lib, lam, h, 1, mode)
    assert np.all(np.isfinite(kap)) and np.all(np.isfinite(F32))
    scale = np.abs(lam).max(axis=1)
    ok = kap >= 1e-3
    err = np.abs(F32 - ref)
    bad = np.nonzero(ok & (err > 1e-4 * np.abs(ref) + 1e-6 * scale))[0]
    assert bad.size == 0, (bad[:5], lam[bad[:5]], F32[bad[:5]], ref[bad[:5]])
    # particles that never collapse get exactly 0
    assert np.all(F32[ref == 0.0][kap[ref == 0.0] >= 1e-3] == 0.0)
    # what goes to the FP64 redo stays rare
    assert (~ok).mean() < 0.02
