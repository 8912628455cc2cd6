"""Served requests on the GPU: concurrent requests overlap on the device and
each result is the same, bit for bit, as the same request run alone."""
import numpy as np
import pytest

from paper_1305_1505_gb300 import ic, serve

pytestmark = pytest.mark.gpu


def test_results_same_alone_and_in_the_mix():
    eng = serve.PinEngine()
    # tile widths tuned per grid size before traffic (kept for the process)
    tiles = eng.warm([16, 32, 48, 64])
    assert sorted(tiles) == [16, 32, 48, 64]
    from paper_1305_1505_gb300 import pin
    for n, (tx, ty) in tiles.items():
        assert tx in pin.pin_tile_options(n) and ty in pin.pin_tile_options(n)
    specs = [(16, 3), (32, 5), (48, 4), (64, 6), (32, 7), (16, 2), (64, 3), (48, 8)]
    reqs = [serve.Request(i, n, 2.0 * n, 500 + i, ic.log_radii(2.0, 20.0, s))
            for i, (n, s) in enumerate(specs)]
    alone = [eng.run(r) for r in reqs]
    srv = serve.Server(eng, budget_bytes=8 * 2 ** 30, max_slots=4)
    mixed = [srv.submit(serve.Request(r.rid, r.n, r.box, r.seed, r.radii)) for r in reqs]
    assert srv.drain(timeout=300)
    srv.close()
    assert srv.peak_running > 1
    for a, m in zip(alone, mixed):
        assert m.status == "done", m.error
        assert np.array_equal(a[0], m.result[0]) and np.array_equal(a[1], m.result[1])
