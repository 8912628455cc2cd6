"""Radius schedule spaced by 0.15 dex in mass variance (Sec. 2.1.1), on the
CPU against the oracle's direct sum over the grid modes."""
import numpy as np
import pytest

import oracle
from paper_1305_1505_gb300 import schedule


@pytest.mark.parametrize("shape,box,r_max", [((16, 16, 16), 64.0, 12.0), ((16, 24, 32), 32.0, 6.0),
                                             ((32, 16, 8), 64.0, 4.0)])
def test_variance_matches_direct_sum(shape, box, r_max):
    v = schedule.Variance(shape, box)
    for R in (0.0, 0.5 * r_max, r_max):
        ref = oracle.sigma2(shape, box, R)
        assert abs(v(R) - ref) <= 1e-12 * ref


@pytest.mark.parametrize("shape,box,r_max", [((16, 16, 16), 64.0, 12.0), ((16, 24, 32), 32.0, 6.0)])
def test_schedule_steps_of_0p15_dex(shape, box, r_max):
    r = schedule.variance_schedule(shape, box, r_max)
    assert r[0] == r_max and np.all(np.diff(r) < 0)
    s2 = np.array([oracle.sigma2(shape, box, x) for x in r])
    assert np.allclose(np.diff(np.log10(s2)), 0.15, rtol=0, atol=1e-10)
    cell = box / shape[0]
    assert r[-1] >= cell
    # the list stops where the next step would go below one cell or past the grid's variance
    nxt = s2[-1] * 10 ** 0.15
    top = oracle.sigma2(shape, box, 0.0)
    assert nxt >= top or oracle.sigma2(shape, box, cell) < nxt


def test_schedule_options():
    r = schedule.variance_schedule((16, 16, 16), 64.0, 12.0, dex=0.3, max_radii=4)
    assert r.size == 4
    r2 = schedule.variance_schedule((16, 16, 16), 64.0, 12.0, r_min=6.0)
    assert r2[-1] >= 6.0 and r2.size < schedule.variance_schedule((16, 16, 16), 64.0, 12.0).size
