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
