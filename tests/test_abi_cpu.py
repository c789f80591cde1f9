"""CPU-side checks of the C ABI: the library builds for sm_103a, loads, exports
every function that include/dugks.h declares, and rejects invalid arguments
before touching a device (no compute call needs a GPU here)."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_1802_02868_gb300 import build, dugks
from paper_1802_02868_gb300 import inputs as I

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if h.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", h)).read()
            names += re.findall(r"^\s*(?:int|void|const char\s*\*)\s*\*?\s*(dugks_\w+)\s*\(", txt, re.M)
    return sorted(set(names))


def test_library_exports_every_declared_symbol():
    lib = ctypes.CDLL(build.build())
    names = declared_functions()
    assert "dugks_step" in names and len(names) >= 18
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_header():
    assert set(dugks.EXPORTS) <= set(declared_functions())


def _args(nx=4, ny=4, **kw):
    m = I.uniform_mesh(nx, ny)
    p = I.Params(beta=0.003, kappa=0.006)
    for k, v in kw.items():
        setattr(p, k, v)
    return m, p


@pytest.mark.parametrize("bad", [dict(nx=0), dict(cfl=0.0), dict(cfl=1.5), dict(phiA=0.0), dict(rhoA=-1.0),
                                 dict(nuB=0.0), dict(tau_g=0.0), dict(mobility=-0.1), dict(beta=float("nan")),
                                 dict(rhoA=2.0, rhoB=1.0, phiA=1.0, phiB=0.5), dict(wall_ny=1), dict(dx0=0.0)])
def test_invalid_arguments_rejected_before_device_work(bad):
    bad = dict(bad)
    nx = bad.pop("nx", 4)
    m, p = _args(nx=max(nx, 1))
    if nx == 0:
        m = I.Mesh(np.zeros(0), np.ones(4))
    if bad.pop("wall_ny", None):
        m = I.Mesh(np.ones(4), np.ones(1), I.PERIODIC, I.WALL)
    if "dx0" in bad:
        bad.pop("dx0")
        m.dx[0] = 0.0
    for k, v in bad.items():
        setattr(p, k, v)
    with pytest.raises(dugks.DugksError) as e:
        dugks.Sim(m, p)
    assert e.value.rc == -1


def test_status_strings():
    assert dugks.status_str(0) == "ok"
    assert dugks.status_str(-3) == "non-finite state"


def test_set_allocator_needs_both_callbacks():
    """dugks_set_allocator takes an alloc/release pair or neither (host-only
    check; nothing is allocated)."""
    L = dugks.load()
    alloc = dugks.ALLOC_FN(lambda n, st, ctx: None)
    assert L.dugks_set_allocator(alloc, dugks.FREE_FN(), None) == -1
    assert L.dugks_set_allocator(dugks.ALLOC_FN(), dugks.FREE_FN(), None) == 0
    dugks.set_allocator(lambda n, st: 0, lambda p, st: None)
    dugks.set_allocator()
    assert dugks._allocator is None


def test_async_conservation_rejects_null_arguments():
    """dugks_conservation_async / _wait check their pointers before any device
    call (host-only)."""
    L = dugks.load()
    assert L.dugks_conservation_async(None, None) == -1
    assert L.dugks_conservation_wait(None) == -1


def test_default_tile_shape_rule_on_the_host():
    """dugks_default_tile_shape, the rule dugks_batch_create applies: the
    16-block strip at >= 3 strips of 16 blocks (32 x 128 cells) per resident
    slot, else the 8-block strip at >= 2 strips of 8 blocks (32 x 64 cells)
    per slot, else the 32x8 tile.  A GB300 has 152 SMs: 304 FP32 slots (two
    strip blocks per SM), 152 FP64 slots.  Strip counts worked out by hand."""
    m = I.uniform_mesh
    f32, f64 = dugks.FP32, dugks.FP64
    assert dugks.default_tile_shape([m(256, 1024)], f32) == 0      # 8 x 8 = 64 of 16; 8 x 16 = 128 of 8
    assert dugks.default_tile_shape([m(1024, 1024)], f32) == 0     # 32 x 8 = 256 < 912; 32 x 16 = 512 < 608
    assert dugks.default_tile_shape([m(1536, 1536)], f32) == 4     # 48 x 12 = 576 < 912; 48 x 24 = 1152
    assert dugks.default_tile_shape([m(2048, 2048)], f32) == 5     # 64 x 16 = 1024 >= 912
    assert dugks.default_tile_shape([m(1024, 1024)], f64) == 4     # 256 < 456; 512 >= 304
    assert dugks.default_tile_shape([m(2048, 2048)], f64) == 5
    assert dugks.default_tile_shape([m(512, 512)], f64) == 0       # 16 x 8 = 128 of 8 < 304
    # the thresholds themselves: a 32 x 128 mesh is one strip of 16 and two of 8
    assert dugks.default_tile_shape([m(32, 128)] * 912, f32) == 5
    assert dugks.default_tile_shape([m(32, 128)] * 911, f32) == 4
    assert dugks.default_tile_shape([m(32, 128)] * 304, f32) == 4
    assert dugks.default_tile_shape([m(32, 128)] * 303, f32) == 0
    # ragged sizes round up: 33 x 129 is 2 x 2 strips of 16 and 2 x 3 of 8
    assert dugks.default_tile_shape([m(33, 129)] * 228, f32) == 5  # 912 strips of 16
    assert dugks.default_tile_shape([m(33, 129)] * 102, f32) == 4  # 408 of 16, 612 of 8
    assert dugks.default_tile_shape([m(33, 129)] * 101, f32) == 0  # 606 of 8
    # another device size scales the slots
    assert dugks.default_tile_shape([m(1024, 1024)], f32, n_sm=64) == 4   # 512 >= 256 of 8, 256 < 384 of 16
    assert dugks.default_tile_shape([m(1024, 1024)], f32, n_sm=32) == 5   # 256 >= 192


def test_default_tile_shape_rejects_bad_arguments():
    L = dugks.load()
    nx = (ctypes.c_int * 1)(64)
    ny = (ctypes.c_int * 1)(64)
    k = ctypes.c_int()
    assert L.dugks_default_tile_shape(nx, ny, 1, dugks.FP32, 0, ctypes.byref(k)) == -1
    assert L.dugks_default_tile_shape(nx, ny, 0, dugks.FP32, 152, ctypes.byref(k)) == -1
    assert L.dugks_default_tile_shape(nx, ny, 1, 7, 152, ctypes.byref(k)) == -1
    assert L.dugks_default_tile_shape(None, ny, 1, dugks.FP32, 152, ctypes.byref(k)) == -1
    zero = (ctypes.c_int * 1)(0)
    assert L.dugks_default_tile_shape(zero, ny, 1, dugks.FP32, 152, ctypes.byref(k)) == -1
    assert L.dugks_default_tile_shape(nx, ny, 1, dugks.FP32, 152, ctypes.byref(k)) == 0 and k.value == 0
