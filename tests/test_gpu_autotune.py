"""The x/y tile schedule (pin_tile_options, pin_set_tiles, pin_autotune):
every candidate width gives bit-identical results (each column's line
transform is the same arithmetic whatever the tile), the tuner picks among
the candidates and keeps its choice per grid shape, and a bad width is
rejected without changing the plan."""
import itertools

import numpy as np
import pytest

from paper_1305_1505_gb300 import ic, pin
from tests import parity

pytestmark = pytest.mark.gpu


def _run(plan, vel=False):
    """Every product that goes through the x/y passes: collapse times, the
    deformation tensor, the Zel'dovich and second-order displacements (and
    v_max with velocities)."""
    F, I = plan.collapse_times()
    out = [F.clone(), I.clone(), plan.hessian(1).clone(), plan.displacements().clone(),
           plan.displacements_2lpt().clone()]
    if vel:
        out.append(plan.velocities().clone())
    return out


@pytest.mark.parametrize("shape,vel", [(32, False), (64, True), (128, False), (384, False),
                                       ((64, 48, 32), True)])
def test_every_tile_width_gives_identical_results(shape, vel):
    import torch
    nx, ny, nz = pin.grid_shape(shape)
    box = 2.0 * nx
    radii = ic.log_radii(2.0, box * min(nx, ny, nz) / nx / 4, 4)
    if nx == ny == nz:
        d32, _ = parity.inputs(nx, box, 21)
    else:
        g = torch.Generator().manual_seed(21)
        d32 = torch.fft.rfftn(torch.randn((nx, ny, nz), generator=g, dtype=torch.float64)).to(torch.complex64)
    plan = pin.Plan(shape, box, radii, velocities=vel)
    try:
        plan.set_ic(torch.as_tensor(d32).cuda())
        assert plan.tiles() == (pin.pin_tile_options(nx)[0], pin.pin_tile_options(ny)[0])
        ref = _run(plan, vel)
        for tx, ty in itertools.product(pin.pin_tile_options(nx), pin.pin_tile_options(ny)):
            plan.set_tiles(tx, ty)
            assert plan.tiles() == (tx, ty)
            got = _run(plan, vel)
            for a, b in zip(ref, got):
                assert torch.equal(a, b), (shape, tx, ty)
        tuned = plan.autotune(reps=2, force=True)
        assert tuned == plan.tiles()
        assert tuned[0] in pin.pin_tile_options(nx) and tuned[1] in pin.pin_tile_options(ny)
        for a, b in zip(ref, _run(plan, vel)):
            assert torch.equal(a, b)
    finally:
        plan.close()


def test_tuner_keeps_its_choice_and_rejects_bad_widths():
    import torch
    n, box = 64, 128.0
    radii = ic.log_radii(2.0, 16.0, 3)
    d32, _ = parity.inputs(n, box, 22)
    a = pin.Plan(n, box, radii)
    b = pin.Plan(n, box, radii)
    try:
        # no field set yet: the tuner runs on a zeroed Phi0
        first = a.autotune(reps=2, force=True)
        # the second plan of the same shape takes the kept choice
        assert b.autotune(reps=2) == first
        before = b.tiles()
        with pytest.raises(pin.PinError) as e:
            b.set_tiles(7, 0)
        assert e.value.status == pin.PIN_EINVAL and b.tiles() == before
        b.set_tiles(0, 0)
        assert b.tiles() == (pin.pin_tile_options(n)[0],) * 2
        # results after tuning equal the default schedule's
        for p in (a, b):
            p.set_ic(torch.from_numpy(d32).cuda())
        Fa, Ia = a.collapse_times()
        Fb, Ib = b.collapse_times()
        assert torch.equal(Fa, Fb) and torch.equal(Ia, Ib)
    finally:
        a.close()
        b.close()


def test_tuner_refuses_inside_stream_capture():
    """Timing cannot happen while the plan's stream records a graph: the call
    returns PIN_ESTATE without enqueuing anything."""
    import torch
    s = torch.cuda.Stream()
    plan = pin.Plan(32, 64.0, [4.0, 2.0], stream=s)
    try:
        x = torch.zeros(8, device="cuda")
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            x.add_(1.0)
            with pytest.raises(pin.PinError) as e:
                plan.autotune(force=True)
        assert e.value.status == pin.PIN_ESTATE
        g.replay()
        torch.cuda.synchronize()
        assert float(x.sum()) == 8.0
        assert plan.autotune(reps=2, force=True) == plan.tiles()
    finally:
        plan.close()
