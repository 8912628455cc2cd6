"""Seeded synthetic Gaussian initial conditions delta(k) (ctypes binding of
ic/pin_ic.c, declared in include/pin_ic.h).

This is the one module that both the CUDA path and the CPU oracle are fed
from: it produces inputs only and holds none of the collapse-time arithmetic.
"""
import ctypes

import numpy as np

from .. import build as _build


class Spectrum(ctypes.Structure):
    _fields_ = [("ns", ctypes.c_double), ("gamma", ctypes.c_double),
                ("sigma8", ctypes.c_double)]


DEFAULT_SPECTRUM = dict(ns=0.96, gamma=0.21, sigma8=0.8)

_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.ensure_ic()
        L = ctypes.CDLL(path)
        sp = ctypes.POINTER(Spectrum)
        L.pin_ic_bbks.argtypes = [ctypes.c_double]
        L.pin_ic_bbks.restype = ctypes.c_double
        L.pin_ic_amplitude.argtypes = [sp]
        L.pin_ic_amplitude.restype = ctypes.c_double
        L.pin_ic_power.argtypes = [ctypes.c_double, sp, ctypes.c_double]
        L.pin_ic_power.restype = ctypes.c_double
        L.pin_ic_delta_k.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_uint64, sp,
                                     ctypes.POINTER(ctypes.c_double)]
        L.pin_ic_delta_k_f32.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_uint64, sp,
                                         ctypes.POINTER(ctypes.c_float)]
        L.pin_ic_splitmix64.argtypes = [ctypes.c_uint64]
        L.pin_ic_splitmix64.restype = ctypes.c_uint64
        _lib = L
    return _lib


def _spec(spectrum):
    s = dict(DEFAULT_SPECTRUM)
    if spectrum:
        s.update(spectrum)
    return Spectrum(s["ns"], s["gamma"], s["sigma8"])


def delta_k(n, box, seed, spectrum=None, dtype=np.complex64):
    """Half-spectrum delta(k), shape (n, n, n//2+1), complex64 or complex128."""
    sp = _spec(spectrum)
    shape = (n, n, n // 2 + 1)
    if np.dtype(dtype) == np.complex128:
        out = np.empty(shape, dtype=np.complex128)
        rc = lib().pin_ic_delta_k(n, box, seed, ctypes.byref(sp),
                                  out.view(np.float64).ctypes.data_as(
                                      ctypes.POINTER(ctypes.c_double)))
    else:
        out = np.empty(shape, dtype=np.complex64)
        rc = lib().pin_ic_delta_k_f32(n, box, seed, ctypes.byref(sp),
                                      out.view(np.float32).ctypes.data_as(
                                          ctypes.POINTER(ctypes.c_float)))
    if rc != 0:
        raise ValueError("pin_ic_delta_k: invalid arguments (n=%r, box=%r)" % (n, box))
    return out


def amplitude(spectrum=None):
    sp = _spec(spectrum)
    return lib().pin_ic_amplitude(ctypes.byref(sp))


def power(k, spectrum=None, amp=None):
    sp = _spec(spectrum)
    a = amplitude(spectrum) if amp is None else amp
    return np.array([lib().pin_ic_power(float(kk), ctypes.byref(sp), a)
                     for kk in np.atleast_1d(k)])


def bbks(q):
    return lib().pin_ic_bbks(q)


def splitmix64(x):
    return lib().pin_ic_splitmix64(x)


def log_radii(r_min, r_max, nscales):
    """Radii log-spaced between r_min and r_max, LARGEST FIRST (index 0 is the
    largest smoothing radius, the order of the trajectory in Sec. 2.1.1)."""
    s = np.arange(nscales, dtype=np.float64)
    if nscales == 1:
        return np.array([float(r_max)])
    r = r_min * (r_max / r_min) ** (s / (nscales - 1))
    return r[::-1].copy()
