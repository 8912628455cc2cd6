"""FP64 CPU oracle of the PINOCCHIO collapse-time step (Sec. 2.1.1).

TEST INFRASTRUCTURE ONLY: imported by tests/, by __graft_entry__.smoke() and
by bench.py's cpu_baseline / reference leg.  The product path never imports
it.  Everything here is argument marshalling around oracle/pin_oracle.c,
except fragment_order (Sec. 2.1.2) and the 2LPT source and its transform in
displacement_2lpt, a few lines of numpy.
"""
import ctypes
import os

import numpy as np

from . import build as _build

_lib = None
_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)


def _p(a, ct=ctypes.c_double):
    return a.ctypes.data_as(ctypes.POINTER(ct)) if a is not None else None


def lib():
    global _lib
    if _lib is None:
        if _build.needs_build():
            p = _build.build()
            if p is not None:
                out, _ = p.communicate()
                if p.returncode != 0:
                    raise RuntimeError("oracle build failed:\n" + out.decode())
        L = ctypes.CDLL(_build.LIB)
        L.or_dft1d.argtypes = [_dp, ctypes.c_int, ctypes.c_int, _dp]
        L.or_idft3d.argtypes = [_dp, ctypes.c_int]
        L.or_hessian.argtypes = [_dp, ctypes.c_int, ctypes.c_double, ctypes.c_double, _dp, _dp]
        L.or_hessian_point.argtypes = [_dp, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                       ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int]
        L.or_hessian_point.restype = ctypes.c_double
        L.or_displacement.argtypes = [_dp, ctypes.c_int, ctypes.c_double, _dp]
        L.or_displacement_r.argtypes = [_dp, ctypes.c_int, ctypes.c_double, ctypes.c_double, _dp]
        L.or_hessian_points.argtypes = [_dp, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                        ctypes.c_int, ctypes.POINTER(ctypes.c_longlong), _dp]
        L.or_hessian3.argtypes = [_dp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                  ctypes.c_double, _dp, _dp]
        L.or_displacement3.argtypes = [_dp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                       ctypes.c_double, _dp]
        L.or_collapse_times3.argtypes = [_dp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                         ctypes.c_int, _dp, ctypes.c_int, _dp, _ip, _dp, _dp, _ip, _dp,
                                         _dp, _dp]
        L.or_collapse_interval.argtypes = [_dp, _dp, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                           ctypes.c_double, _dp, _dp]
        L.or_eig3.argtypes = [_dp, _dp]
        L.or_axis_coeffs.argtypes = [_dp, ctypes.c_int, _dp]
        L.or_first_root.argtypes = [_dp]
        L.or_first_root.restype = ctypes.c_double
        L.or_delta_c.restype = ctypes.c_double
        L.or_x3.restype = ctypes.c_double
        L.or_collapse_F.argtypes = [_dp, ctypes.c_int]
        L.or_collapse_F.restype = ctypes.c_double
        L.or_collapse_point.argtypes = [_dp, ctypes.c_int, _dp]
        L.or_collapse_point.restype = ctypes.c_double
        L.or_collapse_slope.argtypes = [_dp]
        L.or_collapse_slope.restype = ctypes.c_double
        L.or_collapse_times.argtypes = [_dp, ctypes.c_int, ctypes.c_double, ctypes.c_int, _dp,
                                        ctypes.c_int, _dp, _ip, _dp, _dp, _ip, _dp, _dp]
        L.or_collapse_times_sampled.argtypes = [_dp, ctypes.c_int, ctypes.c_double, ctypes.c_int,
                                                _dp, ctypes.c_int, ctypes.c_int,
                                                ctypes.POINTER(ctypes.c_longlong), _dp, _ip, _dp,
                                                _ip]
        L.or_collapse_from_hessians.argtypes = [_dp, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                                _dp, _ip, _dp, _ip]
        _lib = L
    return _lib


def _c128(a):
    return np.ascontiguousarray(a, dtype=np.complex128)


def _grid(half):
    """(nx, ny, nz) of a half-spectrum of shape (nx, ny, nz/2 + 1), nz even."""
    nx, ny, nh = half.shape
    return nx, ny, 2 * (nh - 1)


def dft1d(x, sign=+1):
    """Unnormalised 1D DFT with exp(sign 2 pi i jk/n)."""
    x = _c128(x)
    out = np.empty_like(x)
    lib().or_dft1d(_p(x.view(np.float64)), x.size, sign, _p(out.view(np.float64)))
    return out


def idft3d(a):
    """Normalised inverse 3D DFT of a full complex cube (copy)."""
    a = _c128(a).copy()
    lib().or_idft3d(_p(a.view(np.float64)), a.shape[0])
    return a


def hessian(delta_half, box, radius):
    """(6, nx, ny, nz) FP64 deformation tensor xx, yy, zz, xy, xz, yz, and the
    largest imaginary residue of the inverse transforms (cubic cells: box is
    the side along x)."""
    d = _c128(delta_half)
    nx, ny, nz = _grid(d)
    out = np.empty((6, nx, ny, nz), dtype=np.float64)
    mi = ctypes.c_double()
    rc = lib().or_hessian3(_p(d.view(np.float64)), nx, ny, nz, box, radius, _p(out), ctypes.byref(mi))
    if rc:
        raise ValueError("or_hessian failed: %d" % rc)
    return out, mi.value


def displacement(delta_half, box, radius=0.0):
    """(3, nx, ny, nz) FP64 Zel'dovich displacement psi = i k W(kR) delta / k^2."""
    d = _c128(delta_half)
    nx, ny, nz = _grid(d)
    out = np.empty((3, nx, ny, nz), dtype=np.float64)
    rc = lib().or_displacement3(_p(d.view(np.float64)), nx, ny, nz, box, radius, _p(out))
    if rc:
        raise ValueError("or_displacement failed: %d" % rc)
    return out


def hessian_point(delta_half, box, radius, comp, q):
    d = _c128(delta_half)
    return lib().or_hessian_point(_p(d.view(np.float64)), d.shape[0], box, radius, comp,
                                  int(q[0]), int(q[1]), int(q[2]))


def hessian_points(delta_half, box, radius, q_list):
    """(npts, 6) Hessian components at flat grid indices q by direct summation."""
    d = _c128(delta_half)
    q = np.ascontiguousarray(q_list, dtype=np.int64)
    out = np.empty((q.size, 6))
    rc = lib().or_hessian_points(_p(d.view(np.float64)), d.shape[0], box, radius, q.size,
                                 _p(q, ctypes.c_longlong), _p(out))
    if rc:
        raise ValueError("or_hessian_points failed: %d" % rc)
    return out


def eig3(h6):
    h = np.ascontiguousarray(h6, dtype=np.float64)
    lam = np.empty(3)
    lib().or_eig3(_p(h), _p(lam))
    return lam


def axis_coeffs(lam, i):
    lam = np.ascontiguousarray(lam, dtype=np.float64)
    c = np.empty(3)
    lib().or_axis_coeffs(_p(lam), i, _p(c))
    return c


def first_root(c):
    c = np.ascontiguousarray(c, dtype=np.float64)
    return lib().or_first_root(_p(c))


def delta_c():
    return lib().or_delta_c()


def x3():
    return lib().or_x3()


def collapse_F(lam, correction=1):
    lam = np.ascontiguousarray(lam, dtype=np.float64)
    return lib().or_collapse_F(_p(lam), correction)


def collapse_point(h6, correction=1):
    h = np.ascontiguousarray(h6, dtype=np.float64)
    lam = np.empty(3)
    F = lib().or_collapse_point(_p(h), correction, _p(lam))
    return F, lam


def collapse_slope(lam):
    lam = np.ascontiguousarray(lam, dtype=np.float64)
    return lib().or_collapse_slope(_p(lam))


def collapse_times(delta_half, box, radii, correction=1, keep_all=False, velocities=False):
    """Returns dict with fmax, idx (n^3), f2/idx2 (runner-up), slope, hrms (S:
    the grid's rms tensor norm at each radius), f_all (S, n^3) when keep_all,
    and vmax (3, n^3: the smoothed displacement at the radius of F_max) when
    velocities."""
    d = _c128(delta_half)
    nx, ny, nz = _grid(d)
    r = np.ascontiguousarray(radii, dtype=np.float64)
    S = r.size
    n3 = nx * ny * nz
    fmax = np.empty(n3)
    idx = np.empty(n3, dtype=np.int32)
    f2 = np.empty(n3)
    idx2 = np.empty(n3, dtype=np.int32)
    slope = np.empty(n3)
    f_all = np.empty((S, n3)) if keep_all else None
    vmax = np.empty((3, n3)) if velocities else None
    hrms = np.empty(S)
    rc = lib().or_collapse_times3(_p(d.view(np.float64)), nx, ny, nz, box, S, _p(r), correction,
                                 _p(fmax), _p(idx, ctypes.c_int), _p(f_all), _p(f2),
                                 _p(idx2, ctypes.c_int), _p(slope), _p(vmax), _p(hrms))
    if rc:
        raise ValueError("or_collapse_times failed: %d" % rc)
    out = dict(fmax=fmax, idx=idx, f2=f2, idx2=idx2, slope=slope, hrms=hrms)
    if keep_all:
        out["f_all"] = f_all
    if velocities:
        out["vmax"] = vmax
    return out


def collapse_times_sampled(delta_half, box, radii, q_list, correction=1):
    d = _c128(delta_half)
    n = d.shape[0]
    r = np.ascontiguousarray(radii, dtype=np.float64)
    q = np.ascontiguousarray(q_list, dtype=np.int64)
    m = q.size
    fmax, f2 = np.empty(m), np.empty(m)
    idx, idx2 = np.empty(m, dtype=np.int32), np.empty(m, dtype=np.int32)
    rc = lib().or_collapse_times_sampled(_p(d.view(np.float64)), n, box, r.size, _p(r),
                                         correction, m, _p(q, ctypes.c_longlong), _p(fmax),
                                         _p(idx, ctypes.c_int), _p(f2), _p(idx2, ctypes.c_int))
    if rc:
        raise ValueError("or_collapse_times_sampled failed: %d" % rc)
    return dict(fmax=fmax, idx=idx, f2=f2, idx2=idx2)


def collapse_from_hessians(h6s, correction=1):
    """h6s: (S, npts, 6) Hessians -> running max over S by the oracle."""
    h = np.ascontiguousarray(h6s, dtype=np.float64)
    S, m, _ = h.shape
    fmax, f2 = np.empty(m), np.empty(m)
    idx, idx2 = np.empty(m, dtype=np.int32), np.empty(m, dtype=np.int32)
    lib().or_collapse_from_hessians(_p(h), S, m, correction, _p(fmax), _p(idx, ctypes.c_int),
                                    _p(f2), _p(idx2, ctypes.c_int))
    return dict(fmax=fmax, idx=idx, f2=f2, idx2=idx2)


def collapse_interval(h6s, hscale, u, correction=1):
    """h6s: (S, npts, 6) Hessians, hscale: (S,) rms tensor norms -> (lo, hi),
    each (S, npts): the range of F over eigenvalue errors of half-width
    u (hscale[s] + max |lambda|) (or_collapse_interval)."""
    h = np.ascontiguousarray(h6s, dtype=np.float64)
    S, m, _ = h.shape
    hs = np.ascontiguousarray(hscale, dtype=np.float64)
    if hs.size != S:
        raise ValueError("hscale needs one value per radius")
    lo, hi = np.empty((S, m)), np.empty((S, m))
    lib().or_collapse_interval(_p(h), _p(hs), S, m, correction, float(u), _p(lo), _p(hi))
    return lo, hi


def hessians_at(delta_half, box, radii, q_list):
    """(S, npts, 6) Hessians at flat particle indices q for every radius: the
    direct sum over modes for cubic grids, the full transform otherwise."""
    d = _c128(delta_half)
    nx, ny, nz = _grid(d)
    q = np.ascontiguousarray(q_list, dtype=np.int64)
    out = np.empty((len(radii), q.size, 6))
    for s, R in enumerate(radii):
        if nx == ny == nz:
            out[s] = hessian_points(d, box, R, q)
        else:
            h, _ = hessian(d, box, R)
            out[s] = h.reshape(6, -1)[:, q].T
    return out


def fragment_order(F_max):
    """Fragmentation front end (Sec. 2.1.2) on an (nx, ny, nz) F_max field.
    The particles are considered in descending F_max; equal values in
    ascending particle index q = (x ny + y) nz + z (a reading: the paper
    states no tie rule).  Returns (order, n_before): order[i] is the q of the i-th
    particle considered; n_before[q] counts the six periodic neighbours of q
    (+-1 along each axis) whose rank in that order is below q's.  numpy's
    lexsort and roll serve as the sort and the shifts."""
    F = np.asarray(F_max, dtype=np.float64)
    flat = F.ravel()
    q = np.arange(flat.size)
    order = np.lexsort((q, -flat))  # last key is the primary one
    rank = np.empty(flat.size, dtype=np.int64)
    rank[order] = q
    R = rank.reshape(F.shape)
    n_before = np.zeros(F.shape, dtype=np.int64)
    for axis in range(3):
        for shift in (1, -1):
            n_before += np.roll(R, shift, axis=axis) < R
    return order, n_before


def displacement_2lpt(delta_half, box):
    """Second-order LPT displacement of the unsmoothed field (the standard
    second-order Lagrangian perturbation theory result): with phi_ij the
    deformation tensor at R = 0, S = sum_{i<j} (phi_ii phi_jj - phi_ij^2) and
    psi2(k) = (3/7) i k S(k) / k^2.  The Hessian and the final displacement are
    the C oracle's; numpy's rfftn is the forward transform of S (same sign and
    normalisation convention as delta(k))."""
    h, _ = hessian(delta_half, box, 0.0)
    xx, yy, zz, xy, xz, yz = h
    S = xx * yy + xx * zz + yy * zz - xy ** 2 - xz ** 2 - yz ** 2
    Sk = np.fft.rfftn(S)
    return displacement((3.0 / 7.0) * Sk, box, 0.0)


def sigma2(shape, box, radius, power=None):
    """Variance of the Gaussian-smoothed field on an nx x ny x nz grid with
    cubic cells (box is the side along x), as the radius schedule reads
    Sec. 2.1.1: V^-1 sum over every mode k != 0 of the grid of
    P(k) exp(-k^2 R^2).  power: P(k) for an array of k (default: the power
    spectrum of the initial conditions).  A direct sum over all modes."""
    from paper_1305_1505_gb300 import ic
    nx, ny, nz = shape
    L = [box, box * ny / nx, box * nz / nx]
    k = [2 * np.pi * (np.arange(n) - n // 2) / Li for n, Li in zip(shape, L)]
    k2 = k[0][:, None, None] ** 2 + k[1][None, :, None] ** 2 + k[2][None, None, :] ** 2
    kk = np.sqrt(k2.ravel())
    nz_mask = kk > 0
    P = np.zeros(kk.size)
    P[nz_mask] = (ic.power(kk[nz_mask]) if power is None else power(kk[nz_mask]))
    return float(np.sum(P * np.exp(-k2.ravel() * radius * radius)) / (L[0] * L[1] * L[2]))
