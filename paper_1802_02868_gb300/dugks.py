"""ctypes binding of ``libdugks.so`` (the C ABI of ``include/dugks.h``).

Argument marshalling only: every step of the scheme runs in the library's CUDA
kernels.  The binding raises if the library is missing or a call fails; there
is no fallback of any kind.

``Sim`` wraps one simulation or one batch.  Meshes and parameters are the
``inputs.Mesh`` / ``inputs.Params`` records; fields are numpy float64 arrays
of shape ``[ny, nx]`` (one instance) or lists of them (a batch).  The CUDA
stream is the caller's (``torch.cuda.current_stream().cuda_stream`` or 0).
"""
from __future__ import annotations

import atexit
import ctypes
import os
import weakref

import numpy as np

from . import build as _build

FP64 = 0
FP32 = 1
Q = 9

STATUS = {0: "ok", -1: "invalid argument", -2: "CUDA error", -3: "non-finite state", -4: "out of device memory",
          -5: "device wait timed out", -6: "unsupported"}


class DugksError(RuntimeError):
    def __init__(self, fn, rc):
        super().__init__("%s failed: %s (%d)" % (fn, STATUS.get(rc, "?"), rc))
        self.rc = rc


class NonFiniteError(DugksError):
    pass


class Mesh_t(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("dx", ctypes.POINTER(ctypes.c_double)),
                ("dy", ctypes.POINTER(ctypes.c_double)), ("bc_x", ctypes.c_int), ("bc_y", ctypes.c_int)]


DIAG_FIELDS = ("mass", "xc", "yc", "ux", "uy", "p_bulk_A", "p_bulk_B", "front_y", "tip_y")


class Params_t(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in ("phiA", "phiB", "rhoA", "rhoB", "nuA", "nuB", "mobility", "tau_g",
                                               "beta", "kappa", "gx", "gy", "rho_ref", "cfl")] + \
               [("precision", ctypes.c_int)]


ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p)
_allocator = None          # the callbacks in use (kept alive while sims may call them)
_allocator_sims = []       # weak references to sims that use them, closed at exit


def set_allocator(alloc=None, release=None):
    """Device memory for the sims created from now on: ``alloc(nbytes, stream)``
    returns a device pointer (int, 0 on failure) and ``release(ptr, stream)``
    frees it (dugks_set_allocator); with no arguments cudaMalloc/cudaFree
    come back."""
    global _allocator
    if alloc is None:
        _check("dugks_set_allocator", load().dugks_set_allocator(ALLOC_FN(), FREE_FN(), None))
        _allocator = None
        return

    def _a(n, stream, ctx):
        try:
            return int(alloc(int(n), stream or 0)) or None
        except Exception:
            return None

    def _f(p, stream, ctx):
        try:
            release(int(p), stream or 0)
        except Exception:
            pass

    cb = (ALLOC_FN(_a), FREE_FN(_f))
    _check("dugks_set_allocator", load().dugks_set_allocator(cb[0], cb[1], None))
    _allocator = cb


def use_torch_allocator():
    """Take the device memory of new sims from PyTorch's caching allocator."""
    import torch

    def alloc(n, stream):
        return torch.cuda.caching_allocator_alloc(n, torch.cuda.current_device(), stream)

    def release(p, stream):
        torch.cuda.caching_allocator_delete(p)

    set_allocator(alloc, release)


def _close_allocator_sims():
    for ref in _allocator_sims:
        sim = ref()
        if sim is not None:
            sim.close()


atexit.register(_close_allocator_sims)


class Diag_t(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in DIAG_FIELDS]


_lib = None
EXPORTS = ("dugks_create", "dugks_batch_create", "dugks_destroy", "dugks_init", "dugks_step", "dugks_moments",
           "dugks_conservation", "dugks_conservation_async", "dugks_conservation_wait", "dugks_batch_status", "dugks_dt", "dugks_info", "dugks_save", "dugks_load",
           "dugks_launch_count", "dugks_set_timing", "dugks_kernel_times", "dugks_kernel_name",
           "dugks_kernel_bytes_per_cell", "dugks_status_str", "dugks_conservation_static",
           "dugks_autotune", "dugks_set_tile_shape", "dugks_tile_shape", "dugks_tile_shape_name", "dugks_default_tile_shape",
           "dugks_adjoint", "dugks_uniform_instances", "dugks_diagnostics", "dugks_laplace_pressure",
           "dugks_batch_set_paused", "dugks_batch_step_each", "dugks_set_allocator", "dugks_measure_alu_peaks")
STATIC_MAX_CELLS = 16777216


def library_path():
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libdugks.so (building it with nvcc first if it is missing)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_build.LIB):
        if not build_if_missing:
            raise OSError("libdugks.so is not built: run paper_1802_02868_gb300.build.build()")
        _build.build()
    L = ctypes.CDLL(_build.LIB)
    vp, ip, dp = ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_double)
    L.dugks_create.argtypes = [ctypes.POINTER(Mesh_t), ctypes.POINTER(Params_t), vp, ctypes.POINTER(vp)]
    L.dugks_batch_create.argtypes = [ip, ctypes.POINTER(Mesh_t), ctypes.POINTER(Params_t), vp, ctypes.POINTER(vp)]
    L.dugks_destroy.argtypes = [vp]
    L.dugks_destroy.restype = None
    L.dugks_init.argtypes = [vp, dp, dp, dp, dp]
    L.dugks_step.argtypes = [vp, ctypes.c_long]
    L.dugks_moments.argtypes = [vp, dp, dp, dp, dp, dp]
    L.dugks_conservation.argtypes = [vp, dp, dp]
    L.dugks_conservation_async.argtypes = [vp, dp]
    L.dugks_conservation_wait.argtypes = [vp]
    L.dugks_batch_status.argtypes = [vp, ctypes.POINTER(ctypes.c_int)]
    L.dugks_dt.argtypes = [vp, ip, dp]
    L.dugks_info.argtypes = [vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_long),
                             ctypes.POINTER(ctypes.c_size_t)]
    L.dugks_save.argtypes = [vp, vp, ctypes.POINTER(ctypes.c_size_t)]
    L.dugks_load.argtypes = [vp, vp, ctypes.c_size_t]
    L.dugks_launch_count.argtypes = [vp, ctypes.POINTER(ctypes.c_long)]
    L.dugks_set_timing.argtypes = [vp, ip]
    L.dugks_kernel_times.argtypes = [vp, dp, ctypes.POINTER(ctypes.c_long)]
    L.dugks_kernel_name.argtypes = [ip]
    L.dugks_kernel_name.restype = ctypes.c_char_p
    L.dugks_kernel_bytes_per_cell.argtypes = [vp, ip, dp]
    L.dugks_conservation_static.argtypes = [vp, vp, vp, ip, ip] + [ctypes.c_double] * 4 + [vp, vp]
    L.dugks_adjoint.argtypes = [vp, ctypes.c_long, ip, dp, dp, dp, dp, dp]
    L.dugks_autotune.argtypes = [vp, ip, ctypes.POINTER(ctypes.c_int), dp]
    L.dugks_set_tile_shape.argtypes = [vp, ip]
    L.dugks_tile_shape.argtypes = [vp] + [ctypes.POINTER(ctypes.c_int)] * 3
    L.dugks_uniform_instances.argtypes = [vp, ctypes.POINTER(ctypes.c_int)]
    L.dugks_diagnostics.argtypes = [vp, ctypes.POINTER(Diag_t)]
    L.dugks_laplace_pressure.argtypes = [vp, dp]
    L.dugks_batch_set_paused.argtypes = [vp, ctypes.POINTER(ctypes.c_int)]
    L.dugks_batch_step_each.argtypes = [vp, ctypes.POINTER(ctypes.c_long)]
    L.dugks_set_allocator.argtypes = [ALLOC_FN, FREE_FN, vp]
    L.dugks_measure_alu_peaks.argtypes = [ip, ip, dp, dp, dp, vp]
    L.dugks_tile_shape_name.argtypes = [ip]
    L.dugks_default_tile_shape.argtypes = [ctypes.POINTER(ctypes.c_int)] * 2 + [ip, ip, ip, ctypes.POINTER(ctypes.c_int)]
    L.dugks_tile_shape_name.restype = ctypes.c_char_p
    L.dugks_status_str.argtypes = [ip]
    L.dugks_status_str.restype = ctypes.c_char_p
    for n in EXPORTS:
        if n not in ("dugks_destroy", "dugks_kernel_name", "dugks_status_str", "dugks_tile_shape_name"):
            getattr(L, n).restype = ctypes.c_int
    _lib = L
    return L


NUM_KERNELS = 8


def _check(fn, rc):
    if rc == -3:
        raise NonFiniteError(fn, rc)
    if rc != 0:
        raise DugksError(fn, rc)


def _dp(a):
    return None if a is None else a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a, n):
    a = np.ascontiguousarray(a, dtype=np.float64).reshape(-1)
    if a.size != n:
        raise ValueError("expected %d values, got %d" % (n, a.size))
    return a


class Sim:
    """One simulation (``meshes`` a single Mesh) or a batch (a list of Mesh)."""

    def __init__(self, meshes, params, precision=FP64, stream=0):
        L = load()
        single = not isinstance(meshes, (list, tuple))
        self.meshes = [meshes] if single else list(meshes)
        self.params = [params] * len(self.meshes) if not isinstance(params, (list, tuple)) else list(params)
        if len(self.params) != len(self.meshes):
            raise ValueError("one Params per mesh")
        self.single = single
        n = len(self.meshes)
        self._keep = []
        M = (Mesh_t * n)()
        Pr = (Params_t * n)()
        for k, (m, p) in enumerate(zip(self.meshes, self.params)):
            dx = np.ascontiguousarray(m.dx, dtype=np.float64)
            dy = np.ascontiguousarray(m.dy, dtype=np.float64)
            self._keep += [dx, dy]
            M[k] = Mesh_t(int(dx.size), int(dy.size), _dp(dx), _dp(dy), int(m.bc_x), int(m.bc_y))
            vals = p.as_list()
            Pr[k] = Params_t(*vals, int(precision))
        h = ctypes.c_void_p()
        rc = L.dugks_batch_create(n, M, Pr, ctypes.c_void_p(int(stream)), ctypes.byref(h))
        _check("dugks_batch_create", rc)
        self.h = h
        # a sim created with caller callbacks keeps them alive, and is closed at
        # exit while they still can run
        self._allocator = _allocator
        if _allocator is not None:
            _allocator_sims.append(weakref.ref(self))
        self.precision = precision
        self.sizes = [m.nx * m.ny for m in self.meshes]
        self.ncells = int(sum(self.sizes))

    # -- lifetime
    def close(self):
        if getattr(self, "h", None) and self.h.value:
            load().dugks_destroy(self.h)
            self.h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # -- helpers
    def _cat(self, fields):
        if fields is None:
            return None
        if self.single or (isinstance(fields, np.ndarray) and fields.size == self.ncells):
            return _f64(fields, self.ncells)
        return _f64(np.concatenate([np.asarray(f, dtype=np.float64).reshape(-1) for f in fields]), self.ncells)

    def _split(self, flat):
        out, o = [], 0
        for m, n in zip(self.meshes, self.sizes):
            out.append(flat[o:o + n].reshape(m.ny, m.nx))
            o += n
        return out[0] if self.single else out

    # -- ABI calls
    def init(self, phi, ux=None, uy=None, p=None):
        arrs = [self._cat(phi), self._cat(ux), self._cat(uy), self._cat(p)]
        _check("dugks_init", load().dugks_init(self.h, *[_dp(a) for a in arrs]))
        return self

    def step(self, n=1):
        _check("dugks_step", load().dugks_step(self.h, int(n)))
        return self

    def moments(self, out=None):
        """phi, rho, ux, uy, p of every cell.  ``out``: five flat contiguous
        float64 arrays of all cells (for instance views of pinned host memory)
        that receive the fields directly."""
        if out is None:
            out = [np.zeros(self.ncells) for _ in range(5)]
        else:
            out = list(out)
            for a in out:
                if a.dtype != np.float64 or a.size != self.ncells or not a.flags.c_contiguous:
                    raise ValueError("moments(out=...): five contiguous float64 arrays of %d cells" % self.ncells)
        _check("dugks_moments", load().dugks_moments(self.h, *[_dp(a) for a in out]))
        return dict(zip(("phi", "rho", "ux", "uy", "p"), [self._split(a) for a in out]))

    def conservation(self):
        n = len(self.meshes)
        a, b = np.zeros(n), np.zeros(n)
        _check("dugks_conservation", load().dugks_conservation(self.h, _dp(a), _dp(b)))
        return (a[0], b[0]) if self.single else (a, b)

    def conservation_async(self, sums):
        """dugks_conservation_async: enqueue the FP64 sums into `sums`, a
        page-locked float64 array of 2 n_instances values (sum phi, sum rho
        per instance), and return at once; read it after conservation_wait."""
        n = len(self.meshes)
        if sums.dtype != np.float64 or sums.size != 2 * n or not sums.flags.c_contiguous:
            raise ValueError("sums must be a C-contiguous float64 array of %d values" % (2 * n))
        _check("dugks_conservation_async", load().dugks_conservation_async(self.h, _dp(sums)))
        return sums

    def conservation_wait(self):
        """dugks_conservation_wait: block until the latest conservation_async
        has landed (the stream keeps running what was enqueued after it)."""
        _check("dugks_conservation_wait", load().dugks_conservation_wait(self.h))

    def status(self):
        n = len(self.meshes)
        st = (ctypes.c_int * n)()
        _check("dugks_batch_status", load().dugks_batch_status(self.h, st))
        return list(st)

    def dt(self, k=0):
        v = ctypes.c_double()
        _check("dugks_dt", load().dugks_dt(self.h, int(k), ctypes.byref(v)))
        return v.value

    def state(self):
        """Tracked tilde state as FP64 arrays (f, g), each [9, cells]."""
        nb = ctypes.c_size_t(0)
        _check("dugks_save", load().dugks_save(self.h, None, ctypes.byref(nb)))
        buf = np.zeros(nb.value // 8)
        _check("dugks_save", load().dugks_save(self.h, buf.ctypes.data_as(ctypes.c_void_p), ctypes.byref(nb)))
        buf = buf.reshape(2, Q, self.ncells)
        if self.single:
            m = self.meshes[0]
            return buf[0].reshape(Q, m.ny, m.nx), buf[1].reshape(Q, m.ny, m.nx)
        return buf[0], buf[1]

    def set_state(self, f, g):
        buf = np.ascontiguousarray(np.stack([np.asarray(f, dtype=np.float64).reshape(Q, -1),
                                             np.asarray(g, dtype=np.float64).reshape(Q, -1)]))
        if buf.shape[2] != self.ncells:
            raise ValueError("state has %d cells, expected %d" % (buf.shape[2], self.ncells))
        _check("dugks_load", load().dugks_load(self.h, buf.ctypes.data_as(ctypes.c_void_p), buf.nbytes))

    def set_paused(self, paused):
        """Pause (True) or resume (False) each instance (dugks_batch_set_paused)."""
        n = len(self.meshes)
        arr = (ctypes.c_int * n)(*[1 if p else 0 for p in paused])
        _check("dugks_batch_set_paused", load().dugks_batch_set_paused(self.h, arr))
        return self

    def step_each(self, nsteps):
        """Advance instance k by nsteps[k] steps (dugks_batch_step_each)."""
        n = len(self.meshes)
        arr = (ctypes.c_long * n)(*[int(v) for v in nsteps])
        _check("dugks_batch_step_each", load().dugks_batch_step_each(self.h, arr))
        return self

    def diagnostics_array(self, out=None):
        """dugks_diagnostics into an (instances, 9) float64 array (columns in
        DIAG_FIELDS order, the layout of dugks_diag); `out` may be given."""
        n = len(self.meshes)
        if out is None:
            out = np.empty((n, len(DIAG_FIELDS)))
        if out.shape != (n, len(DIAG_FIELDS)) or out.dtype != np.float64 or not out.flags.c_contiguous:
            raise ValueError("out must be a C-contiguous float64 array of shape (%d, %d)" % (n, len(DIAG_FIELDS)))
        _check("dugks_diagnostics", load().dugks_diagnostics(self.h, out.ctypes.data_as(ctypes.POINTER(Diag_t))))
        return out

    def diagnostics(self):
        """Per-instance diagnostics (dugks_diagnostics) as dicts; one dict for a
        single instance."""
        ds = [dict(zip(DIAG_FIELDS, row)) for row in self.diagnostics_array().tolist()]
        return ds[0] if self.single else ds

    def laplace_pressure(self):
        """The Laplace pressure field P of every instance (dugks_laplace_pressure)."""
        out = np.zeros(self.ncells)
        _check("dugks_laplace_pressure", load().dugks_laplace_pressure(self.h, _dp(out)))
        return self._split(out)

    def uniform_instances(self):
        """Instances on the fused step's uniform periodic path."""
        v = ctypes.c_int()
        _check("dugks_uniform_instances", load().dugks_uniform_instances(self.h, ctypes.byref(v)))
        return v.value

    def launch_count(self):
        v = ctypes.c_long()
        _check("dugks_launch_count", load().dugks_launch_count(self.h, ctypes.byref(v)))
        return v.value

    def set_timing(self, on=True):
        _check("dugks_set_timing", load().dugks_set_timing(self.h, 1 if on else 0))

    def kernel_times(self):
        ms = np.zeros(NUM_KERNELS)
        n = (ctypes.c_long * NUM_KERNELS)()
        _check("dugks_kernel_times", load().dugks_kernel_times(self.h, _dp(ms), n))
        return {kernel_name(k): (ms[k], n[k]) for k in range(NUM_KERNELS)}

    def adjoint(self, nsteps, phi_target, ckpt_every=100):
        """Gradient of L = sum_cells (phi_T - phi_target)^2 after ``nsteps`` steps
        from the last ``init`` inputs, by the library's reverse sweep with
        checkpoints every ``ckpt_every`` steps.  Returns a dict with ``loss``,
        ``dphi0`` (field(s) like the init phi), ``dkappa`` and ``dlambda``
        (per instance for a batch, scalars for one simulation)."""
        n = len(self.meshes)
        tgt = self._cat(phi_target)
        loss, dk, dl = np.zeros(n), np.zeros(n), np.zeros(n)
        dphi = np.zeros(self.ncells)
        _check("dugks_adjoint", load().dugks_adjoint(self.h, int(nsteps), int(ckpt_every), _dp(tgt), _dp(loss),
                                                      _dp(dphi), _dp(dk), _dp(dl)))
        if self.single:
            return {"loss": loss[0], "dphi0": self._split(dphi), "dkappa": dk[0], "dlambda": dl[0]}
        return {"loss": loss, "dphi0": self._split(dphi), "dkappa": dk, "dlambda": dl}

    def autotune(self, steps=5):
        """Time every tile shape of the fused step on the current state (which is
        restored) and keep the fastest; returns (shape index, name, ms per step)."""
        k = ctypes.c_int()
        ms = ctypes.c_double()
        _check("dugks_autotune", load().dugks_autotune(self.h, int(steps), ctypes.byref(k), ctypes.byref(ms)))
        return k.value, tile_shape_name(k.value), ms.value

    def set_tile_shape(self, shape):
        _check("dugks_set_tile_shape", load().dugks_set_tile_shape(self.h, int(shape)))

    def tile_shape(self):
        k, bx, by = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        _check("dugks_tile_shape", load().dugks_tile_shape(self.h, ctypes.byref(k), ctypes.byref(bx), ctypes.byref(by)))
        return k.value, bx.value, by.value

    def kernel_bytes_per_cell(self, k):
        v = ctypes.c_double()
        _check("dugks_kernel_bytes_per_cell", load().dugks_kernel_bytes_per_cell(self.h, int(k), ctypes.byref(v)))
        return v.value


def conservation_static(phi_ptr, dx_ptr, dy_ptr, nx, ny, params, out_ptr, stream=0):
    """Allocation-free conservation sums of one mesh from caller-owned device
    buffers (raw device addresses): phi[ny][nx], dx[nx], dy[ny] in, out[2] out.
    Returns the status code (0 on success) without raising."""
    return load().dugks_conservation_static(ctypes.c_void_p(int(phi_ptr)), ctypes.c_void_p(int(dx_ptr)),
                                            ctypes.c_void_p(int(dy_ptr)), int(nx), int(ny), params.phiA,
                                            params.phiB, params.rhoA, params.rhoB, ctypes.c_void_p(int(out_ptr)),
                                            ctypes.c_void_p(int(stream)))


def measure_alu_peaks(iters_f32=262144, iters_f64=4096, stream=0):
    """FMA throughput of the current device in TFLOP/s (dugks_measure_alu_peaks):
    a dict with fp32, fp32x2 (packed two-lane FMAs) and fp64."""
    a, b, c = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    _check("dugks_measure_alu_peaks", load().dugks_measure_alu_peaks(int(iters_f32), int(iters_f64), ctypes.byref(a),
                                                                      ctypes.byref(b), ctypes.byref(c),
                                                                      ctypes.c_void_p(int(stream))))
    return {"fp32": a.value, "fp32x2": b.value, "fp64": c.value}


NUM_TILE_SHAPES = 7


def default_tile_shape(meshes, precision=FP32, n_sm=152):
    """dugks_default_tile_shape: the shape a new fused-step sim of these meshes
    starts with on a device of n_sm multiprocessors (no device needed)."""
    meshes = list(meshes) if isinstance(meshes, (list, tuple)) else [meshes]
    nx = (ctypes.c_int * len(meshes))(*[m.nx for m in meshes])
    ny = (ctypes.c_int * len(meshes))(*[m.ny for m in meshes])
    k = ctypes.c_int()
    _check("dugks_default_tile_shape",
           load().dugks_default_tile_shape(nx, ny, len(meshes), int(precision), int(n_sm), ctypes.byref(k)))
    return k.value


def tile_shape_name(k):
    return load().dugks_tile_shape_name(int(k)).decode()


def kernel_name(k):
    return load().dugks_kernel_name(int(k)).decode()


def kernel_name_index(name):
    for k in range(NUM_KERNELS):
        if kernel_name(k) == name:
            return k
    raise KeyError(name)


def status_str(rc):
    return load().dugks_status_str(int(rc)).decode()
