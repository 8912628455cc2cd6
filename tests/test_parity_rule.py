"""The host logic of the parity rule's conditioning clause (tests/parity.py)
on hand-made oracle ranges (CPU only)."""
import numpy as np

from tests import parity


def test_within_conditioning_cases():
    # two particles (columns), three radii (rows)
    lo = np.array([[0.10, 0.00], [0.50, 0.00], [0.20, 0.00]])
    hi = np.array([[0.12, 0.00], [0.70, 0.01], [0.80, 0.00]])
    tol = np.array([1e-3, 1e-3])
    # F_max range of particle 0: [0.50, 0.80]; radius 1 holds [0.50, 0.70],
    # radius 2 [0.20, 0.80], radius 0 [0.10, 0.12]
    F = np.array([0.75, 0.0])
    I = np.array([2, -1])
    assert parity.within_conditioning(F, I, lo, hi, tol).tolist() == [True, True]
    # radius 1 cannot reach 0.75
    assert not parity.within_conditioning(F[:1], np.array([1]), lo[:, :1], hi[:, :1], tol[:1])[0]
    # radius 0 cannot hold the maximum at all
    assert not parity.within_conditioning(np.array([0.11]), np.array([0]), lo[:, :1], hi[:, :1], tol[:1])[0]
    # above the range
    assert not parity.within_conditioning(np.array([0.9]), np.array([2]), lo[:, :1], hi[:, :1], tol[:1])[0]
    # "never collapses" only where the oracle's lower bound allows F_max = 0
    assert not parity.within_conditioning(np.array([0.0]), np.array([-1]), lo[:, :1], hi[:, :1], tol[:1])[0]
    # particle 1 may collapse at radius 1 (hi 0.01) or never
    assert parity.within_conditioning(np.array([0.008]), np.array([1]), lo[:, 1:], hi[:, 1:], tol[1:])[0]
    assert not parity.within_conditioning(np.array([0.008]), np.array([0]), lo[:, 1:], hi[:, 1:], tol[1:])[0]
