"""Python binding of libbgk (include/bgk.h): the same entry points, argument marshalling only.

Every step of the method runs in the CUDA library; this module converts numpy arrays / torch
tensors to pointers and C structs. It raises if the compiled library is missing: there is no
fallback path.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

from . import _build

BGK_OK, BGK_EINVAL, BGK_ENOMEM, BGK_ECUDA, BGK_ENEWTON, BGK_EDOMAIN, BGK_ETIMEOUT = 0, -1, -2, -3, -4, -5, -6
BC_PERIODIC, BC_DIRICHLET, BC_DIFFUSE_WALL, BC_EXCHANGE = 0, 1, 2, 3
FP32_SPLIT, FP64 = 0, 1
MAXWELLIAN_CONSERVATIVE, MAXWELLIAN_CONTINUOUS = 0, 1

# every symbol include/bgk.h declares
SYMBOLS = (
    "bgk_create", "bgk_destroy", "bgk_last_error", "bgk_set_stream", "bgk_info", "bgk_points",
    "bgk_set_state", "bgk_set_state_device", "bgk_set_f", "bgk_get_f", "bgk_step", "bgk_moments",
    "bgk_moments_device", "bgk_equilibrium", "bgk_synchronize", "bgk_dt", "bgk_set_timing", "bgk_timing",
    "bgk_equilibrium_noalloc", "bgk_autotune", "bgk_set_geometry", "bgk_set_connectivity", "bgk_f_distance",
    "bgk_halo_floats", "bgk_halo_pack", "bgk_set_halo", "bgk_stage",
    "bgk_batch_create", "bgk_batch_destroy", "bgk_batch_last_error", "bgk_batch_set_stream", "bgk_batch_step",
    "bgk_batch_synchronize", "bgk_batch_autotune", "bgk_batch_info", "bgk_batch_set_timing", "bgk_batch_timing",
)


class bgk_mesh(C.Structure):
    _fields_ = [("dim", C.c_int), ("nelem", C.c_int * 3), ("lo", C.c_double * 3), ("hi", C.c_double * 3),
                ("bc", (C.c_int * 2) * 3), ("bc_state", ((C.c_double * 5) * 2) * 3)]


class bgk_vgrid(C.Structure):
    _fields_ = [("n", C.c_int * 3), ("lo", C.c_double * 3), ("hi", C.c_double * 3)]


class bgk_opts(C.Structure):
    _fields_ = [("precision", C.c_int), ("body_force", C.c_double * 3), ("newton_max_it", C.c_int),
                ("newton_tol", C.c_double), ("limiter", C.c_int), ("chunks", C.c_int),
                ("vtiles_per_task", C.c_int), ("maxwellian", C.c_int), ("mu_ref", C.c_double),
                ("mu_omega", C.c_double)]


class BgkError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"libbgk error {code}: {msg}")
        self.code = code


_lock = threading.Lock()
_lib = None


def lib_path() -> str:
    return _build.LIB


def lib():
    """Load libbgk.so. Raises if it has not been built (no CPU fallback exists)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(_build.LIB):
                raise RuntimeError(f"libbgk is not built ({_build.LIB} missing): run __graft_entry__.build()")
            L = C.CDLL(_build.LIB)
            vp, dp, i64p = C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_int64)
            L.bgk_create.argtypes = [C.POINTER(bgk_mesh), C.c_int, C.POINTER(bgk_vgrid), C.c_double,
                                     C.POINTER(bgk_opts), C.POINTER(C.c_void_p)]
            L.bgk_destroy.argtypes = [vp]
            L.bgk_destroy.restype = None
            L.bgk_last_error.argtypes = [vp]
            L.bgk_last_error.restype = C.c_char_p
            L.bgk_set_stream.argtypes = [vp, vp]
            L.bgk_info.argtypes = [vp, i64p, i64p, i64p, i64p]
            for name in ("bgk_points", "bgk_set_state", "bgk_set_f", "bgk_get_f", "bgk_moments", "bgk_equilibrium"):
                getattr(L, name).argtypes = [vp, dp]
            L.bgk_set_state_device.argtypes = [vp, vp]
            L.bgk_moments_device.argtypes = [vp, vp]
            L.bgk_step.argtypes = [vp, C.c_double, C.c_int]
            L.bgk_synchronize.argtypes = [vp]
            L.bgk_dt.argtypes = [vp, C.c_double]
            L.bgk_dt.restype = C.c_double
            L.bgk_set_timing.argtypes = [vp, C.c_int]
            L.bgk_timing.argtypes = [vp, dp, i64p, dp, i64p, dp]
            L.bgk_equilibrium_noalloc.argtypes = [vp, C.c_int64, C.POINTER(bgk_vgrid), vp, vp, vp]
            L.bgk_autotune.argtypes = [vp, C.POINTER(C.c_int)]
            L.bgk_f_distance.argtypes = [vp, vp, dp, dp]
            L.bgk_halo_floats.argtypes = [vp, i64p]
            L.bgk_halo_pack.argtypes = [vp, C.c_int, vp, vp]
            L.bgk_set_halo.argtypes = [vp, C.c_int, vp]
            L.bgk_stage.argtypes = [vp, C.c_double, C.c_int]
            L.bgk_set_geometry.argtypes = [vp, C.POINTER(C.c_double)]
            L.bgk_set_connectivity.argtypes = [vp, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int)]
            L.bgk_batch_create.argtypes = [C.c_int, C.POINTER(vp), C.POINTER(vp)]
            L.bgk_batch_destroy.argtypes = [vp]
            L.bgk_batch_destroy.restype = None
            L.bgk_batch_last_error.argtypes = [vp]
            L.bgk_batch_last_error.restype = C.c_char_p
            L.bgk_batch_set_stream.argtypes = [vp, vp]
            L.bgk_batch_step.argtypes = [vp, dp, C.c_int]
            L.bgk_batch_synchronize.argtypes = [vp]
            L.bgk_batch_autotune.argtypes = [vp]
            L.bgk_batch_info.argtypes = [vp, i64p, i64p, i64p]
            L.bgk_batch_set_timing.argtypes = [vp, C.c_int]
            L.bgk_batch_timing.argtypes = [vp, dp, i64p, dp, i64p, dp]
            _lib = L
    return _lib


def _dptr(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def make_mesh(dim, nelem, lo, hi, bc=None, bc_state=None) -> bgk_mesh:
    m = bgk_mesh()
    m.dim = dim
    for d in range(dim):
        m.nelem[d] = int(nelem[d])
        m.lo[d] = float(lo[d])
        m.hi[d] = float(hi[d])
    for d in range(dim, 3):
        m.nelem[d] = 1
        m.lo[d], m.hi[d] = 0.0, 1.0
    if bc is not None:
        b = np.asarray(bc, dtype=np.int32).reshape(3, 2)
        for d in range(3):
            for s in range(2):
                m.bc[d][s] = int(b[d, s])
    if bc_state is not None:
        st = np.asarray(bc_state, dtype=np.float64).reshape(3, 2, 5)
        for d in range(3):
            for s in range(2):
                for q in range(5):
                    m.bc_state[d][s][q] = float(st[d, s, q])
    return m


def make_vgrid(n, lo, hi) -> bgk_vgrid:
    v = bgk_vgrid()
    for d in range(3):
        v.n[d] = int(n[d])
        v.lo[d] = float(lo[d])
        v.hi[d] = float(hi[d])
    return v


def make_opts(precision=FP32_SPLIT, body_force=(0.0, 0.0, 0.0), newton_max_it=0, chunks=0, vtiles_per_task=0,
              limiter=False, maxwellian=0, mu_ref=0.0, mu_omega=0.0):
    """maxwellian: MAXWELLIAN_CONSERVATIVE (the method) or MAXWELLIAN_CONTINUOUS (the ablation)."""
    o = bgk_opts()
    o.precision = precision
    for d in range(3):
        o.body_force[d] = float(body_force[d])
    o.newton_max_it = newton_max_it
    o.newton_tol = 0.0
    o.limiter = int(bool(limiter))
    o.chunks = chunks
    o.vtiles_per_task = vtiles_per_task
    o.maxwellian = int(maxwellian)
    o.mu_ref = float(mu_ref)
    o.mu_omega = float(mu_omega)
    return o


def equilibrium_noalloc(f_dev, nv, vlo, vhi, Q_dev, prim_dev, stream_ptr=None):
    """bgk_equilibrium_noalloc on caller-owned CUDA tensors: f_dev float32 [npts, N_v], Q_dev and
    prim_dev float64 [npts, 5], all on one device. For callers that cannot allocate device memory: the
    library uses only its fixed static scratch. The C entry point cannot see buffer sizes, so every
    shape, dtype and device is checked here and a mismatch raises ValueError before anything is
    launched. stream_ptr defaults to torch's current stream on f's device. Returns the status code
    (0 on success)."""
    import torch

    nvel = int(np.prod([int(x) for x in nv]))
    if f_dev.dtype != torch.float32 or f_dev.dim() != 2 or f_dev.shape[1] != nvel or not f_dev.is_contiguous():
        raise ValueError(f"f must be a contiguous float32 [npts, {nvel}] tensor, got {f_dev.dtype} "
                         f"{tuple(f_dev.shape)}")
    npts = int(f_dev.shape[0])
    for name, t in (("Q", Q_dev), ("prim", prim_dev)):
        if t.dtype != torch.float64 or tuple(t.shape) != (npts, 5) or not t.is_contiguous():
            raise ValueError(f"{name} must be a contiguous float64 [{npts}, 5] tensor, got {t.dtype} {tuple(t.shape)}")
        if t.device != f_dev.device:
            raise ValueError(f"{name} is on {t.device}, f on {f_dev.device}")
    if not f_dev.is_cuda:
        raise ValueError("f, Q and prim must be CUDA tensors")
    if stream_ptr is None:
        stream_ptr = torch.cuda.current_stream(f_dev.device).cuda_stream
    vg = make_vgrid(nv, vlo, vhi)
    return lib().bgk_equilibrium_noalloc(C.c_void_p(f_dev.data_ptr()), npts, C.byref(vg),
                                         C.c_void_p(Q_dev.data_ptr()), C.c_void_p(prim_dev.data_ptr()),
                                         C.c_void_p(stream_ptr or 0))


class Solver:
    """One libbgk context (bgk_create ... bgk_destroy) with numpy/torch marshalling."""

    def __init__(self, dim, nelem, lo, hi, p, nv, vlo, vhi, tau, bc=None, bc_state=None, **opts):
        L = lib()
        self._mesh = make_mesh(dim, nelem, lo, hi, bc, bc_state)
        self._vg = make_vgrid(nv, vlo, vhi)
        self._opts = make_opts(**opts)
        h = C.c_void_p()
        rc = L.bgk_create(C.byref(self._mesh), int(p), C.byref(self._vg), float(tau), C.byref(self._opts), C.byref(h))
        if rc != BGK_OK:
            raise BgkError(rc, "bgk_create failed (see stderr)")
        self.h = h
        n, v, d, b = C.c_int64(), C.c_int64(), C.c_int64(), C.c_int64()
        L.bgk_info(self.h, C.byref(n), C.byref(v), C.byref(d), C.byref(b))
        self.npts, self.nvel, self.ndof, self.device_bytes = n.value, v.value, d.value, b.value

    def _check(self, rc):
        if rc != BGK_OK:
            raise BgkError(rc, lib().bgk_last_error(self.h).decode())

    def close(self):
        if getattr(self, "h", None):
            lib().bgk_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_stream(self, stream_ptr):
        self._check(lib().bgk_set_stream(self.h, C.c_void_p(stream_ptr or 0)))

    def points(self):
        x = np.zeros((self.npts, 3))
        self._check(lib().bgk_points(self.h, _dptr(x)))
        return x

    def set_geometry(self, x):
        """Curvilinear hexahedra: physical coordinates x [n_x, 3] (FP64, host) of every solution node."""
        a = np.ascontiguousarray(x, dtype=np.float64).reshape(self.npts, 3)
        self._check(lib().bgk_set_geometry(self.h, _dptr(a)))

    def set_connectivity(self, nbr, nface, orient):
        """Unstructured hexahedral connectivity: [n_elements, 6] neighbour, shared-face and orientation
        tables (host int arrays)."""
        a = [np.ascontiguousarray(t, dtype=np.int32).reshape(-1) for t in (nbr, nface, orient)]
        ip = C.POINTER(C.c_int)
        self._check(lib().bgk_set_connectivity(self.h, a[0].ctypes.data_as(ip), a[1].ctypes.data_as(ip),
                                               a[2].ctypes.data_as(ip)))

    def set_state(self, prim):
        """prim: numpy (host) or torch tensor [n_x, 5] (rho, u, v, w, T), FP64, host or CUDA."""
        if hasattr(prim, "is_cuda") and prim.is_cuda:
            assert prim.dtype.is_floating_point and prim.element_size() == 8 and prim.is_contiguous()
            self._check(lib().bgk_set_state_device(self.h, C.c_void_p(prim.data_ptr())))
            return
        if hasattr(prim, "data_ptr"):  # torch CPU tensor (possibly pinned)
            assert prim.element_size() == 8 and prim.is_contiguous()
            self._check(lib().bgk_set_state(self.h, C.cast(C.c_void_p(prim.data_ptr()), C.POINTER(C.c_double))))
            return
        a = np.ascontiguousarray(prim, dtype=np.float64).reshape(self.npts, 5)
        self._check(lib().bgk_set_state(self.h, _dptr(a)))

    def set_f(self, f):
        a = np.ascontiguousarray(f, dtype=np.float64).reshape(self.npts, self.nvel)
        self._check(lib().bgk_set_f(self.h, _dptr(a)))

    def get_f(self):
        a = np.zeros((self.npts, self.nvel))
        self._check(lib().bgk_get_f(self.h, _dptr(a)))
        return a

    def step(self, dt, nsteps=1):
        self._check(lib().bgk_step(self.h, float(dt), int(nsteps)))

    def moments(self, out=None):
        """Host FP64 [n_x, 5]; with a CUDA tensor `out`, an asynchronous device copy instead."""
        if out is not None and hasattr(out, "is_cuda") and out.is_cuda:
            self._check(lib().bgk_moments_device(self.h, C.c_void_p(out.data_ptr())))
            return out
        if out is not None and hasattr(out, "data_ptr"):
            self._check(lib().bgk_moments(self.h, C.cast(C.c_void_p(out.data_ptr()), C.POINTER(C.c_double))))
            return out
        Q = np.zeros((self.npts, 5))
        self._check(lib().bgk_moments(self.h, _dptr(Q)))
        return Q

    def equilibrium(self):
        P = np.zeros((self.npts, 5))
        self._check(lib().bgk_equilibrium(self.h, _dptr(P)))
        return P

    def synchronize(self):
        self._check(lib().bgk_synchronize(self.h))

    def dt(self, cfl):
        return lib().bgk_dt(self.h, float(cfl))

    def autotune(self):
        """Pick the fastest task length for this problem (cached per shape); returns it."""
        g = C.c_int()
        self._check(lib().bgk_autotune(self.h, C.byref(g)))
        return g.value

    def set_timing(self, on):
        self._check(lib().bgk_set_timing(self.h, int(bool(on))))

    def halo_floats(self):
        n = C.c_int64()
        self._check(lib().bgk_halo_floats(self.h, C.byref(n)))
        return n.value

    def halo_pack(self, stage, lo=None, hi=None):
        """Enqueue copies of the element layers next to the lo / hi x faces of the source of `stage`
        into the float32 CUDA tensors lo, hi (halo_floats() each; either may be None)."""
        for t in (lo, hi):
            if t is not None:
                assert t.is_cuda and t.dtype.itemsize == 4 and t.is_contiguous() and t.numel() >= self.halo_floats()
        self._check(lib().bgk_halo_pack(self.h, int(stage), C.c_void_p(lo.data_ptr() if lo is not None else 0),
                                        C.c_void_p(hi.data_ptr() if hi is not None else 0)))

    def set_halo(self, face, t):
        """The neighbour's layer across x face 0 (lo) or 1 (hi): a float32 CUDA tensor of halo_floats(),
        read by the stage kernel while it is set (None: the context's own zero halo)."""
        if t is not None:
            assert t.is_cuda and t.dtype.itemsize == 4 and t.is_contiguous() and t.numel() >= self.halo_floats()
        self._halo = getattr(self, "_halo", [None, None])
        self._halo[face] = t  # kept alive while the library reads it
        self._check(lib().bgk_set_halo(self.h, int(face), C.c_void_p(t.data_ptr() if t is not None else 0)))

    def stage(self, dt, stage):
        """Enqueue stage `stage` (0, 1, 2) of one SSP-RK3 step."""
        self._check(lib().bgk_stage(self.h, float(dt), int(stage)))

    def f_distance(self, other):
        """(max |f_self - f_other|, max |f_other|) over every real degree of freedom, on the device."""
        d, m = C.c_double(), C.c_double()
        self._check(lib().bgk_f_distance(self.h, other.h, C.byref(d), C.byref(m)))
        return d.value, m.value

    def timing(self):
        sm, nm, by = C.c_double(), C.c_double(), C.c_double()
        sl, nl = C.c_int64(), C.c_int64()
        self._check(lib().bgk_timing(self.h, C.byref(sm), C.byref(sl), C.byref(nm), C.byref(nl), C.byref(by)))
        return dict(stage_ms=sm.value, stage_launches=sl.value, newton_ms=nm.value, newton_launches=nl.value,
                    stage_alg_bytes=by.value)


class Batch:
    """A batch of Solver members stepped together (bgk_batch_create ... bgk_batch_destroy).
    Members must be FP32-split line problems created with chunks=1; the batch does not own them."""

    def __init__(self, members):
        L = lib()
        self.members = list(members)
        arr = (C.c_void_p * len(self.members))(*[m.h for m in self.members])
        h = C.c_void_p()
        rc = L.bgk_batch_create(len(self.members), arr, C.byref(h))
        if rc != BGK_OK:
            raise BgkError(rc, "bgk_batch_create failed (see stderr)")
        self.h = h
        n, d, t = C.c_int64(), C.c_int64(), C.c_int64()
        L.bgk_batch_info(self.h, C.byref(n), C.byref(d), C.byref(t))
        self.npts, self.ndof, self.tasks = n.value, d.value, t.value

    def _check(self, rc):
        if rc != BGK_OK:
            raise BgkError(rc, lib().bgk_batch_last_error(self.h).decode())

    def close(self):
        if getattr(self, "h", None):
            lib().bgk_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_stream(self, stream_ptr):
        self._check(lib().bgk_batch_set_stream(self.h, C.c_void_p(stream_ptr or 0)))

    def step(self, dt, nsteps=1):
        """dt: one time step per member (sequence of floats)."""
        a = np.ascontiguousarray(dt, dtype=np.float64)
        assert a.shape == (len(self.members),)
        self._dt = a  # the library reads it during the call only
        self._check(lib().bgk_batch_step(self.h, _dptr(a), int(nsteps)))

    def synchronize(self):
        self._check(lib().bgk_batch_synchronize(self.h))

    def autotune(self):
        self._check(lib().bgk_batch_autotune(self.h))
        n, d, t = C.c_int64(), C.c_int64(), C.c_int64()
        lib().bgk_batch_info(self.h, C.byref(n), C.byref(d), C.byref(t))
        self.tasks = t.value

    def set_timing(self, on):
        self._check(lib().bgk_batch_set_timing(self.h, int(bool(on))))

    def timing(self):
        sm, nm, by = C.c_double(), C.c_double(), C.c_double()
        sl, nl = C.c_int64(), C.c_int64()
        self._check(lib().bgk_batch_timing(self.h, C.byref(sm), C.byref(sl), C.byref(nm), C.byref(nl), C.byref(by)))
        return dict(stage_ms=sm.value, stage_launches=sl.value, newton_ms=nm.value, newton_launches=nl.value,
                    stage_alg_bytes=by.value)
