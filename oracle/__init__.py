"""CPU FP64 oracle of the two-phase DUGKS step -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The CUDA library never does, and this
package never imports the library: the two share nothing but the seeded input
generators.

``build()`` compiles ``dugks_oracle.c`` with gcc (``-ffp-contract=off`` so x86
and Arm produce identical bits; OpenMP over rows when available) into
``oracle/_build/liboracle.so`` and ``Oracle`` wraps it with ctypes.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "dugks_oracle.c")
BUILD_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD_DIR, "liboracle.so")
LIB_CS = os.path.join(BUILD_DIR, "liboracle_cs.so")   # double complex build (complex step)

Q = 9
_lib = None


def _compile(out, defines=()):
    if os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(SRC):
        return out
    base = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off"] + list(defines) + [SRC]
    tmp = out + ".tmp.%d" % os.getpid()
    try:
        subprocess.run(base + ["-fopenmp", "-o", tmp, "-lm"], check=True,
                       stdout=subprocess.PIPE, stderr=subprocess.PIPE)
    except subprocess.CalledProcessError:
        subprocess.run(base + ["-o", tmp, "-lm"], check=True)
    os.replace(tmp, out)
    return out


def build(force: bool = False) -> str:
    """Compile the oracle shared libraries (idempotent): the double build and
    the double-complex build used for complex-step derivatives."""
    os.makedirs(BUILD_DIR, exist_ok=True)
    if force:
        for f in (LIB, LIB_CS):
            if os.path.exists(f):
                os.remove(f)
    _compile(LIB)
    _compile(LIB_CS, ["-DORACLE_COMPLEX"])
    return LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(LIB)
        dp = ctypes.POINTER(ctypes.c_double)
        vp = ctypes.c_void_p
        L.oracle_create.restype = vp
        L.oracle_create.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, dp, dp, dp]
        L.oracle_destroy.argtypes = [vp]
        L.oracle_dt.restype = ctypes.c_double
        L.oracle_dt.argtypes = [vp]
        L.oracle_init.argtypes = [vp, dp, dp, dp, dp]
        L.oracle_init.restype = ctypes.c_int
        L.oracle_step.argtypes = [vp, ctypes.c_long]
        L.oracle_step.restype = ctypes.c_int
        L.oracle_moments.argtypes = [vp, dp, dp, dp, dp, dp]
        L.oracle_aux.argtypes = [vp] + [dp] * 9
        L.oracle_get_state.argtypes = [vp, dp, dp]
        L.oracle_set_state.argtypes = [vp, dp, dp]
        L.oracle_conservation.argtypes = [vp, dp, dp]
        L.oracle_derivatives.argtypes = [vp, dp, dp, dp, dp]
        L.oracle_bar_plus_fields.argtypes = [vp, dp, dp]
        L.oracle_derived.argtypes = [vp, dp]
        L.oracle_feq.argtypes = [ctypes.c_double] * 4 + [dp]
        L.oracle_geq.argtypes = [ctypes.c_double] * 5 + [dp]
        L.oracle_src_f.argtypes = [ctypes.c_double] * 10 + [dp]
        L.oracle_src_g.argtypes = [ctypes.c_double] * 8 + [dp]
        for fn, n in (("oracle_bar_plus", 5), ("oracle_original", 5), ("oracle_tilde_plus", 2)):
            getattr(L, fn).argtypes = [ctypes.c_double] * n
            getattr(L, fn).restype = ctypes.c_double
        L.oracle_width_sigma.argtypes = [ctypes.c_double] * 4 + [dp, dp]
        _lib = L
    return _lib


def _p(a):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _c(a, n=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if n is not None and a.size != n:
        raise ValueError("expected %d values, got %d" % (n, a.size))
    return a


# --- point functions (pins) --------------------------------------------------

def feq(p, rho, ux, uy):
    out = np.zeros(Q)
    lib().oracle_feq(p, rho, ux, uy, _p(out))
    return out


def geq(phi, mu, eta, ux, uy):
    out = np.zeros(Q)
    lib().oracle_geq(phi, mu, eta, ux, uy, _p(out))
    return out


def src_f(ux, uy, Fx, Fy, grx, gry, rho, gamma, lam, lap_mu):
    out = np.zeros(Q)
    lib().oracle_src_f(ux, uy, Fx, Fy, grx, gry, rho, gamma, lam, lap_mu, _p(out))
    return out


def src_g(phi, rho, ux, uy, Fx, Fy, gpx, gpy):
    out = np.zeros(Q)
    lib().oracle_src_g(phi, rho, ux, uy, Fx, Fy, gpx, gpy, _p(out))
    return out


def bar_plus(tilde, eq, src, tau, dt):
    return lib().oracle_bar_plus(tilde, eq, src, tau, dt)


def tilde_plus(bar_plus_value, tilde):
    return lib().oracle_tilde_plus(bar_plus_value, tilde)


def original(bar, eq, src, tau, h):
    return lib().oracle_original(bar, eq, src, tau, h)


def width_sigma(beta, kappa, phiA=1.0, phiB=0.0):
    W = ctypes.c_double()
    s = ctypes.c_double()
    lib().oracle_width_sigma(beta, kappa, phiA, phiB, ctypes.byref(W), ctypes.byref(s))
    return W.value, s.value


# --- a simulation ------------------------------------------------------------

class Oracle:
    """One mesh advanced by the FP64 oracle.  ``mesh`` and ``params`` follow
    ``paper_1802_02868_gb300.inputs`` (duck-typed: dx, dy, bc_x, bc_y and
    ``params.as_list()``)."""

    def __init__(self, mesh, params):
        L = lib()
        self.nx, self.ny = int(mesh.dx.size), int(mesh.dy.size)
        self.N = self.nx * self.ny
        self._dx = _c(mesh.dx)
        self._dy = _c(mesh.dy)
        self._prm = _c(params.as_list(), 14)
        self.h = L.oracle_create(self.nx, self.ny, int(mesh.bc_x), int(mesh.bc_y),
                                 _p(self._dx), _p(self._dy), _p(self._prm))
        if not self.h:
            raise ValueError("oracle_create failed")

    def close(self):
        if self.h:
            lib().oracle_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def dt(self):
        return lib().oracle_dt(self.h)

    def derived(self):
        out = np.zeros(6)
        lib().oracle_derived(self.h, _p(out))
        return dict(zip(("dt", "h", "eta", "gamma", "muA", "muB"), out))

    def init(self, phi, ux=None, uy=None, p=None):
        arrs = [_c(phi, self.N)] + [None if a is None else _c(a, self.N) for a in (ux, uy, p)]
        self._keep = arrs
        rc = lib().oracle_init(self.h, *[_p(a) for a in arrs])
        if rc != 0:
            raise FloatingPointError("oracle_init: non-finite state")
        return self

    def step(self, n=1, check=True):
        rc = lib().oracle_step(self.h, int(n))
        if rc != 0 and check:
            raise FloatingPointError("oracle_step: non-finite state")
        return rc

    def moments(self):
        out = [np.zeros(self.N) for _ in range(5)]
        lib().oracle_moments(self.h, *[_p(a) for a in out])
        shp = (self.ny, self.nx)
        return dict(zip(("phi", "rho", "ux", "uy", "p"), [a.reshape(shp) for a in out]))

    def aux(self):
        """Cell fields of the last macro evaluation (call ``moments`` first)."""
        out = [np.zeros(self.N) for _ in range(9)]
        lib().oracle_aux(self.h, *[_p(a) for a in out])
        shp = (self.ny, self.nx)
        names = ("mu", "lap_mu", "gmux", "gmuy", "gpx", "gpy", "gphix", "gphiy", "tauf")
        return dict(zip(names, [a.reshape(shp) for a in out]))

    def state(self):
        f = np.zeros((Q, self.ny, self.nx))
        g = np.zeros((Q, self.ny, self.nx))
        lib().oracle_get_state(self.h, _p(f), _p(g))
        return f, g

    def set_state(self, f, g):
        f = _c(f, Q * self.N)
        g = _c(g, Q * self.N)
        lib().oracle_set_state(self.h, _p(f), _p(g))

    def conservation(self):
        a = ctypes.c_double()
        b = ctypes.c_double()
        lib().oracle_conservation(self.h, ctypes.byref(a), ctypes.byref(b))
        return a.value, b.value

    def derivatives(self, F):
        F = _c(F, self.N)
        dx, dy, lap = (np.zeros(self.N) for _ in range(3))
        lib().oracle_derivatives(self.h, _p(F), _p(dx), _p(dy), _p(lap))
        shp = (self.ny, self.nx)
        return dx.reshape(shp), dy.reshape(shp), lap.reshape(shp)

    def bar_plus_fields(self):
        fb = np.zeros((Q, self.ny, self.nx))
        gb = np.zeros((Q, self.ny, self.nx))
        lib().oracle_bar_plus_fields(self.h, _p(fb), _p(gb))
        return fb, gb


_lib_cs = None


def lib_cs():
    global _lib_cs
    if _lib_cs is None:
        build()
        L = ctypes.CDLL(LIB_CS)
        dp = ctypes.POINTER(ctypes.c_double)
        vp = ctypes.c_void_p
        L.oracle_create.restype = vp
        L.oracle_create.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, dp, dp, dp]
        L.oracle_destroy.argtypes = [vp]
        L.oracle_init.argtypes = [vp, dp, dp, dp, dp]
        L.oracle_init.restype = ctypes.c_int
        L.oracle_step.argtypes = [vp, ctypes.c_long]
        L.oracle_step.restype = ctypes.c_int
        L.oracle_moments.argtypes = [vp, dp, dp, dp, dp, dp]
        L.oracle_get_state.argtypes = [vp, dp, dp]
        _lib_cs = L
    return _lib_cs


def _cp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


class OracleCS:
    """The oracle in double complex arithmetic, for complex-step derivatives.
    ``params`` is a list of 14 complex numbers in the order of
    ``Params.as_list()`` (the CFL number's real part is used)."""

    def __init__(self, mesh, params_complex):
        L = lib_cs()
        self.nx, self.ny = int(mesh.dx.size), int(mesh.dy.size)
        self.N = self.nx * self.ny
        self._dx = _c(mesh.dx)
        self._dy = _c(mesh.dy)
        self._prm = np.ascontiguousarray(np.asarray(params_complex, dtype=np.complex128).reshape(14))
        self.h = L.oracle_create(self.nx, self.ny, int(mesh.bc_x), int(mesh.bc_y), _p(self._dx), _p(self._dy),
                                 _cp(self._prm))
        if not self.h:
            raise ValueError("oracle_create failed")

    def close(self):
        if self.h:
            lib_cs().oracle_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def init(self, phi):
        self._phi = np.ascontiguousarray(np.asarray(phi, dtype=np.complex128).reshape(-1))
        if lib_cs().oracle_init(self.h, _cp(self._phi), None, None, None) != 0:
            raise FloatingPointError("oracle_init: non-finite state")
        return self

    def step(self, n=1):
        if lib_cs().oracle_step(self.h, int(n)) != 0:
            raise FloatingPointError("oracle_step: non-finite state")
        return self

    def phi(self):
        out = np.zeros(self.N, dtype=np.complex128)
        lib_cs().oracle_moments(self.h, _cp(out), None, None, None, None)
        return out.reshape(self.ny, self.nx)


def complex_step_gradient(mesh, params, phi0, steps, phi_target, direction_phi0=None, which=(), eps=1e-30):
    """Derivatives of L = sum_cells (phi_T - phi_target)^2 by the complex step:
    for each parameter name in ``which`` (``"kappa"`` or ``"mobility"``) dL/dparam,
    and, if ``direction_phi0`` is given, the directional derivative dL/dphi0 . v."""
    names = ("phiA", "phiB", "rhoA", "rhoB", "nuA", "nuB", "mobility", "tau_g", "beta", "kappa", "gx", "gy",
             "rho_ref", "cfl")
    base = np.asarray(params.as_list(), dtype=np.complex128)
    out = {}

    def loss(prm, phi):
        o = OracleCS(mesh, prm).init(phi).step(steps)
        d = o.phi() - phi_target
        return np.sum(d * d)

    for w in which:
        prm = base.copy()
        prm[names.index(w)] += 1j * eps
        out[w] = loss(prm, np.asarray(phi0, dtype=np.complex128)).imag / eps
    if direction_phi0 is not None:
        phi = np.asarray(phi0, dtype=np.complex128) + 1j * eps * np.asarray(direction_phi0)
        out["phi0_dir"] = loss(base, phi).imag / eps
    return out


def run_case(case, steps=None):
    """Convenience: build, initialise and advance a ``inputs.Case``."""
    o = Oracle(case.mesh, case.params)
    o.init(case.phi0, case.ux0, case.uy0, case.p0)
    n = case.steps if steps is None else steps
    if n:
        o.step(n)
    return o
