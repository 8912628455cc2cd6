"""Smoothing radii spaced in mass variance (Sec. 2.1.1: successive radii
differ by a fixed 0.15 dex step in the variance of the smoothed field, and
10 to 20 of them suffice for the trajectories).

Reading: sigma^2(R) is the expected variance of the field smoothed with the
Gaussian window W = exp(-k^2 R^2 / 2) on the simulation grid itself,
    sigma^2(R) = V^-1 sum_{k != 0 on the grid} P(k) exp(-k^2 R^2),
with the power spectrum of the initial conditions; the first radius is the
caller's r_max, each next one raises log10 sigma^2 by `dex`, and the list
stops before a radius below r_min (default: one grid cell) or once the grid's
unsmoothed variance cannot be exceeded.

Host-side (numpy): it runs once per plan, before any device work.  Cells are
cubic (box is the side along x), so k^2 is an integer multiple of
(2 pi / (cell M))^2 with M = lcm(nx, ny, nz); the sum runs over the distinct
integers with their multiplicities (3.2e5 terms at 768^3).
"""
import math

import numpy as np

from . import ic


def _shape(n):
    if np.ndim(n) == 0:
        return (int(n),) * 3
    return tuple(int(v) for v in n)


class Variance:
    """sigma^2(R) of an nx x ny x nz grid with cubic cells (box along x)."""

    def __init__(self, shape, box, spectrum=None):
        nx, ny, nz = _shape(shape)
        self.cell = box / nx
        M = math.lcm(nx, ny, nz)
        # integer coordinates of the squared wavenumbers: k_i = 2 pi m_i / (n_i cell)
        # = (2 pi / (M cell)) (M / n_i) m_i
        sq = []
        for n in (nx, ny, nz):
            m = np.arange(n) - n // 2  # every mode of the full grid, Nyquist included once
            sq.append(((M // n) * m) ** 2)
        vxy = (sq[0][:, None] + sq[1][None, :]).ravel()
        hxy = np.bincount(vxy)
        vmax = int(vxy.max() + sq[2].max())
        hist = np.zeros(vmax + 1, dtype=np.int64)
        for v in sq[2]:
            hist[v:v + hxy.size] += hxy
        hist[0] -= 1  # k = 0 is not part of the field
        v = np.nonzero(hist)[0]
        self.count = hist[v].astype(np.float64)
        self.k2 = (2 * np.pi / (M * self.cell)) ** 2 * v.astype(np.float64)
        self.P = ic.power(np.sqrt(self.k2), spectrum)
        self.volume = nx * ny * nz * self.cell ** 3

    def __call__(self, R):
        return float(np.sum(self.count * self.P * np.exp(-self.k2 * R * R)) / self.volume)

    def with_slope(self, R):
        """(sigma^2(R), d sigma^2 / dR)."""
        t = self.count * self.P * np.exp(-self.k2 * R * R)
        return float(np.sum(t) / self.volume), float(-2.0 * R * np.sum(t * self.k2) / self.volume)


def variance_schedule(shape, box, r_max, r_min=None, dex=0.15, max_radii=64, spectrum=None):
    """Radii (Mpc/h), largest first: r_max, then each next radius with
    log10 sigma^2 larger by `dex`, while the radius stays >= r_min (default
    one cell) and at most max_radii of them."""
    var = Variance(shape, box, spectrum)
    if r_min is None:
        r_min = var.cell
    top = var(0.0)
    radii = [float(r_max)]
    s2 = var(r_max)
    while len(radii) < max_radii:
        target = s2 * 10.0 ** dex
        if target >= top:
            break
        # sigma^2 decreases with R: the root lies in (0, R_prev); Newton on
        # ln sigma^2, kept inside the bracket (bisection when it leaves it)
        lo, hi = 0.0, radii[-1]
        r = radii[-1] * 10.0 ** (-dex / 2)
        for _ in range(100):
            f, df = var.with_slope(r)
            if f > target:
                lo = r
            else:
                hi = r
            g = math.log(f / target)
            step = g / (df / f) if df != 0.0 else 0.0
            nr = r - step
            if not (lo < nr < hi):
                nr = 0.5 * (lo + hi)
            if abs(nr - r) <= 1e-14 * r:
                r = nr
                break
            r = nr
        if r < r_min:
            break
        radii.append(r)
        s2 = var(r)
    return np.array(radii)
