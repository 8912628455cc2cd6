"""The C-ABI libraries load and export every declared symbol; argument
validation works without a GPU (no compute call is made here)."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_1305_1505_gb300 import build, pin

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared(header):
    txt = open(os.path.join(ROOT, "include", header)).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(pin_\w+)\s*\(", txt)))


def test_libpin_exports_every_declared_symbol():
    lib = ctypes.CDLL(build.ensure_pin())
    names = _declared("pin.h")
    assert "pin_plan" in names and "pin_collapse_times" in names and "pin_displacements" in names
    for name in names:
        assert hasattr(lib, name), name
    assert set(pin.EXPORTS) == set(names)


def test_libpin_ic_exports_every_declared_symbol():
    lib = ctypes.CDLL(build.ensure_ic())
    for name in _declared("pin_ic.h"):
        assert hasattr(lib, name), name


def test_validation_without_gpu():
    L = pin.load()
    assert pin.pin_strerror(pin.PIN_EINVAL) == "invalid argument"
    good = pin.make_desc(64, 100.0, [10.0, 5.0])
    assert pin.pin_footprint_bytes(good) > 64 ** 3 * 8
    for bad in (pin.make_desc(60, 100.0, [1.0]),       # unsupported size
                pin.make_desc(64, -1.0, [1.0]),        # bad box
                pin.make_desc(64, 100.0, [-1.0]),      # bad radius
                pin.make_desc(64, 100.0, [np.nan]),
                pin.make_desc(64, 100.0, [1.0] * 65)):  # too many radii
        assert pin.pin_footprint_bytes(bad) == 0
        h = ctypes.c_void_p()
        assert L.pin_plan(ctypes.byref(h), ctypes.byref(bad)) == pin.PIN_EINVAL
        assert not h.value
    nc = pin.make_desc((64, 32, 48), 100.0, [1.0])  # non-cubic grids of supported sizes are valid
    assert pin.pin_footprint_bytes(nc) > 64 * 32 * 48 * 8
    nc = pin.make_desc(64, 100.0, [1.0])
    nc.ny = 60  # one unsupported axis is enough to reject
    assert pin.pin_footprint_bytes(nc) == 0
    nc = pin.make_desc(64, 100.0, [1.0])
    nc.correction = 7
    assert pin.pin_footprint_bytes(nc) == 0


def test_null_plan_calls_are_rejected():
    L = pin.load()
    assert L.pin_set_ic(None, None, 0, 0) == pin.PIN_EINVAL
    assert L.pin_collapse_times(None, None, None, 0) == pin.PIN_EINVAL
    assert L.pin_sync(None, 0) == pin.PIN_EINVAL
    assert L.pin_kernels_per_call(None) == 0
    L.pin_destroy(None)


def test_tile_options_without_gpu():
    """Candidate x/y tile widths: the default first, then half of it while a
    TMA box row stays at least 64 bytes (8 complex values); nothing for an
    unsupported size; the plan-level calls reject a null plan."""
    for n in (8, 16, 32, 48, 64, 96, 128, 192, 256, 384, 512, 768):
        opts = pin.pin_tile_options(n)
        assert 1 <= len(opts) <= 2 and all(t >= 8 for t in opts), (n, opts)
        if len(opts) == 2:
            assert opts[1] * 2 == opts[0], (n, opts)
    assert pin.pin_tile_options(768) == [16, 8]
    with pytest.raises(pin.PinError):
        pin.pin_tile_options(100)
    L = pin.load()
    x = ctypes.c_int(0)
    assert L.pin_get_tiles(None, ctypes.byref(x), ctypes.byref(x)) == pin.PIN_EINVAL
    assert L.pin_set_tiles(None, 0, 0) == pin.PIN_EINVAL
    assert L.pin_autotune(None, 3, 0, None, None) == pin.PIN_EINVAL


def test_more_validation_and_footprint_without_gpu():
    """Batch limits, flag values, missing radii; the footprint grows with the
    batch and with velocities, and at 768^3 matches the workspace the layout
    describes (10 padded spectra, F_max and index, tables, redo queue:
    about 22.2 GB; with velocities 13 spectra and two 3 N^3 float arrays,
    about 38.5 GB)."""
    def fp(d):
        return pin.pin_footprint_bytes(d)
    base = pin.make_desc(768, 3072.0, [120.0, 4.0])
    assert abs(fp(base) / 1e9 - 22.2) < 0.2
    vel = pin.make_desc(768, 3072.0, [120.0, 4.0], velocities=True)
    assert abs(fp(vel) / 1e9 - 38.5) < 0.2
    four = pin.make_desc(768, 3072.0, [120.0, 4.0], batch=4)  # 4 x 768^3 < 2^31
    assert fp(four) > 3.9 * fp(base)
    assert fp(pin.make_desc(768, 3072.0, [1.0], batch=5)) == 0  # 5 x 768^3 >= 2^31
    assert fp(pin.make_desc(8, 16.0, [1.0], batch=4096)) > 0
    assert fp(pin.make_desc(8, 16.0, [1.0], batch=4097)) == 0
    d = pin.make_desc(64, 100.0, [1.0])
    d.velocities = 2
    assert fp(d) == 0
    d = pin.make_desc(64, 100.0, [1.0])
    d.precision = 2
    assert fp(d) == 0
    # PIN_FP64 adds its FP64 workspace: half-spectrum 16 B, complex cube 16 B,
    # tensor 48 B and F_max 8 B per mode / particle; batch 1 only
    d = pin.make_desc(64, 100.0, [1.0], precision=pin.PIN_FP64)
    extra = fp(d) - fp(pin.make_desc(64, 100.0, [1.0]))
    assert extra == 64 * 64 * 33 * 16 + 64 ** 3 * (16 + 48 + 8)
    assert fp(pin.make_desc(64, 100.0, [1.0], precision=pin.PIN_FP64, batch=2)) == 0
    d = pin.make_desc(64, 100.0, [1.0])
    d.radii = None
    assert fp(d) == 0
    d = pin.make_desc(64, 100.0, [1.0])
    d.nscales = 0
    assert fp(d) == 0
    assert fp(pin.make_desc(64, float("inf"), [1.0])) == 0
    assert fp(pin.make_desc(64, 100.0, [0.0])) > 0  # R = 0 (no smoothing) is a valid radius
