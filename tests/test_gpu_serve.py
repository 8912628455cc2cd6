"""Served requests on the GPU: concurrent requests overlap on the device,
each result is the same, bit for bit, as the same request run alone, and the
plan pool serves every request after warm-up without making a plan."""
import numpy as np
import pytest

from paper_1305_1505_gb300 import ic, serve

pytestmark = pytest.mark.gpu


def test_results_same_alone_and_in_the_mix():
    eng = serve.PinEngine(pool_per_size=4)
    # tile widths tuned per grid size before traffic (kept for the process),
    # and the pool filled with plans of each size
    tiles = eng.warm([16, 32, 48, 64], per_size=2)
    assert sorted(tiles) == [16, 32, 48, 64]
    from paper_1305_1505_gb300 import pin
    for n, ((tx, ty), (vx, vy)) in tiles.items():
        assert tx in pin.pin_tile_options_radix(n, vx) and ty in pin.pin_tile_options_radix(n, vy)
    specs = [(16, 3), (32, 5), (48, 4), (64, 6), (32, 7), (16, 2), (64, 3), (48, 8)]
    reqs = [serve.Request(i, n, 2.0 * n, 500 + i, ic.log_radii(2.0, 20.0, s))
            for i, (n, s) in enumerate(specs)]
    alone = []
    for r in reqs:
        F, I, release = eng.run(r)
        alone.append((F.copy(), I.copy()))
        release()
    made = eng.plans_made
    srv = serve.Server(eng, budget_bytes=8 * 2 ** 30, max_slots=4)
    mixed = [srv.submit(serve.Request(r.rid, r.n, r.box, r.seed, r.radii)) for r in reqs]
    assert srv.drain(timeout=300)
    srv.close()
    assert srv.peak_running > 1
    for a, m in zip(alone, mixed):
        assert m.status == "done", m.error
        assert np.array_equal(a[0], m.result[0]) and np.array_equal(a[1], m.result[1])
    # at most two requests of a size ran at once and two plans per size were
    # warm: no plan was made during the traffic
    assert eng.plans_made == made, (made, eng.plans_made)
    eng.close()
