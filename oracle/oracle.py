"""Python handle on the FP64 CPU oracle (``oracle/bgk_oracle.c``).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` use it to check and time the CUDA library. It compiles the C oracle with gcc into
``oracle/_build/`` and calls it through ctypes. It imports nothing from the CUDA package.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "liborc.so")
SRC = os.path.join(HERE, "bgk_oracle.c")

PERIODIC, DIRICHLET, WALL, EXCHANGE = 0, 1, 2, 3

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle (gcc, -O2, OpenMP) unless an up-to-date build exists."""
    os.makedirs(BUILD, exist_ok=True)
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= max(
        os.path.getmtime(SRC), os.path.getmtime(os.path.join(HERE, "bgk_oracle.h"))
    ):
        return LIB
    tmp = LIB + f".tmp{os.getpid()}"
    subprocess.check_call(
        ["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", "-Wall", "-o", tmp, SRC, "-lm"]
    )
    os.replace(tmp, LIB)
    return LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(LIB)
            dp = C.POINTER(C.c_double)
            ip = C.POINTER(C.c_int)
            L.oracle_gauss_legendre.argtypes = [C.c_int, dp, dp]
            L.oracle_fr_operators.argtypes = [C.c_int, dp, dp, dp, dp, dp]
            L.oracle_velocity_grid.argtypes = [ip, dp, dp, dp, dp]
            L.oracle_create.restype = C.c_void_p
            L.oracle_create.argtypes = [C.c_int, ip, dp, dp, ip, dp, C.c_int, ip, dp, dp, C.c_double, dp]
            L.oracle_destroy.argtypes = [C.c_void_p]
            L.oracle_npoints.restype = C.c_int64
            L.oracle_npoints.argtypes = [C.c_void_p]
            L.oracle_nvel.restype = C.c_int64
            L.oracle_nvel.argtypes = [C.c_void_p]
            for name in ("oracle_points", "oracle_set_state", "oracle_set_f", "oracle_get_f",
                         "oracle_moments"):
                getattr(L, name).argtypes = [C.c_void_p, dp]
            L.oracle_moments_of.argtypes = [C.c_void_p, dp, dp]
            L.oracle_residual.argtypes = [C.c_void_p, dp, dp]
            L.oracle_rhs.argtypes = [C.c_void_p, dp, dp]
            L.oracle_conservative_maxwellian.argtypes = [C.c_void_p, C.c_int64, dp, dp, ip, dp]
            L.oracle_sample_maxwellian.argtypes = [C.c_void_p, dp, dp]
            L.oracle_step.argtypes = [C.c_void_p, C.c_double, C.c_int]
            L.oracle_dt.restype = C.c_double
            L.oracle_dt.argtypes = [C.c_void_p, C.c_double]
            L.oracle_set_newton.argtypes = [C.c_void_p, C.c_double, C.c_int]
            L.oracle_set_maxwellian.argtypes = [C.c_void_p, C.c_int]
            L.oracle_set_limiter.argtypes = [C.c_void_p, C.c_int]
            L.oracle_limit.argtypes = [C.c_void_p, dp]
            L.oracle_set_viscosity.argtypes = [C.c_void_p, C.c_double, C.c_double]
            L.oracle_set_geometry.argtypes = [C.c_void_p, dp]
            L.oracle_metric.argtypes = [C.c_void_p, dp, dp]
            L.oracle_set_connectivity.argtypes = [C.c_void_p, ip, ip, ip]
            L.oracle_stage.argtypes = [C.c_void_p, C.c_double, C.c_int]
            L.oracle_pack_halo.argtypes = [C.c_void_p, C.c_int, C.c_int, dp]
            L.oracle_set_halo.argtypes = [C.c_void_p, C.c_int, dp]
            _lib = L
    return _lib


def _d(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _i(a):
    return a.ctypes.data_as(C.POINTER(C.c_int))


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


def gauss_legendre(n: int):
    x = np.zeros(n)
    w = np.zeros(n)
    assert lib().oracle_gauss_legendre(n, _d(x), _d(w)) == 0
    return x, w


def fr_operators(p: int):
    n = p + 1
    D = np.zeros((n, n))
    lm, lp, dgl, dgr = (np.zeros(n) for _ in range(4))
    assert lib().oracle_fr_operators(p, _d(D), _d(lm), _d(lp), _d(dgl), _d(dgr)) == 0
    return D, lm, lp, dgl, dgr


def velocity_grid(nv, vlo, vhi):
    nv = np.asarray(nv, dtype=np.int32)
    n = int(np.prod(nv))
    xi = np.zeros((n, 3))
    w = np.zeros(n)
    assert lib().oracle_velocity_grid(_i(nv), _d(_f64(vlo)), _d(_f64(vhi)), _d(xi), _d(w)) == 0
    return xi, w


class Problem:
    """One oracle problem: mesh, velocity grid, relaxation time, boundary data and the state f."""

    def __init__(self, dim, nelem, lo, hi, p, nv, vlo, vhi, tau, bc=None, bc_state=None, force=None):
        L = lib()
        self.dim, self.p = dim, p
        ne = np.zeros(3, np.int32)
        ne[:dim] = nelem[:dim]
        lo_ = np.zeros(3)
        hi_ = np.ones(3)
        lo_[:dim] = lo[:dim]
        hi_[:dim] = hi[:dim]
        bc_ = np.zeros(6, np.int32) if bc is None else np.asarray(bc, np.int32).reshape(6)
        bs_ = np.zeros(30) if bc_state is None else _f64(bc_state, (30,))
        nv_ = np.asarray(nv, np.int32)
        fz = None if force is None else _f64(force, (3,))
        self._keep = (ne, lo_, hi_, bc_, bs_, nv_, fz)
        self.h = L.oracle_create(dim, _i(ne), _d(lo_), _d(hi_), _i(bc_), _d(bs_), p, _i(nv_),
                                 _d(_f64(vlo)), _d(_f64(vhi)), float(tau),
                                 None if fz is None else _d(fz))
        if not self.h:
            raise ValueError("oracle_create rejected the problem")
        self.npts = L.oracle_npoints(self.h)
        self.nvel = L.oracle_nvel(self.h)
        self.xi, self.w = velocity_grid(nv, vlo, vhi)

    def __del__(self):
        h = getattr(self, "h", None)
        if h:
            lib().oracle_destroy(h)
            self.h = None

    def points(self):
        x = np.zeros((self.npts, 3))
        lib().oracle_points(self.h, _d(x))
        return x

    def set_state(self, prim):
        prim = _f64(prim, (self.npts, 5))
        rc = lib().oracle_set_state(self.h, _d(prim))
        if rc != 0:
            raise ValueError(f"oracle_set_state: {rc}")

    def set_f(self, f):
        f = _f64(f, (self.npts, self.nvel))
        assert lib().oracle_set_f(self.h, _d(f)) == 0

    def get_f(self):
        f = np.zeros((self.npts, self.nvel))
        assert lib().oracle_get_f(self.h, _d(f)) == 0
        return f

    def moments(self, f=None):
        Q = np.zeros((self.npts, 5))
        if f is None:
            lib().oracle_moments(self.h, _d(Q))
        else:
            f = _f64(f, (self.npts, self.nvel))
            lib().oracle_moments_of(self.h, _d(f), _d(Q))
        return Q

    def residual(self, f):
        f = _f64(f, (self.npts, self.nvel))
        R = np.zeros_like(f)
        assert lib().oracle_residual(self.h, _d(f), _d(R)) == 0
        return R

    def rhs(self, f):
        f = _f64(f, (self.npts, self.nvel))
        Lf = np.zeros_like(f)
        rc = lib().oracle_rhs(self.h, _d(f), _d(Lf))
        if rc != 0:
            raise RuntimeError(f"oracle_rhs: {rc}")
        return Lf

    def conservative_maxwellian(self, Q):
        Q = _f64(Q)
        Q2 = Q.reshape(-1, 5)
        n = Q2.shape[0]
        P = np.zeros((n, 5))
        it = np.zeros(n, np.int32)
        res = np.zeros(n)
        bad = lib().oracle_conservative_maxwellian(self.h, n, _d(Q2), _d(P), _i(it), _d(res))
        return P.reshape(Q.shape), it, res, bad

    def sample_maxwellian(self, prim):
        g = np.zeros(self.nvel)
        rc = lib().oracle_sample_maxwellian(self.h, _d(_f64(prim, (5,))), _d(g))
        if rc != 0:
            raise ValueError("bad Maxwellian state")
        return g

    def step(self, dt, nsteps=1):
        rc = lib().oracle_step(self.h, float(dt), int(nsteps))
        if rc != 0:
            raise RuntimeError(f"oracle_step: {rc}")

    def dt(self, cfl):
        return lib().oracle_dt(self.h, float(cfl))

    def set_newton(self, tol, max_it):
        lib().oracle_set_newton(self.h, float(tol), int(max_it))

    def set_maxwellian(self, continuous):
        """False: the discretely-conservative Maxwellian; True: the continuous one of Q (ablation)."""
        lib().oracle_set_maxwellian(self.h, int(bool(continuous)))

    def set_viscosity(self, mu_ref, omega):
        """tau = mu_ref theta^omega / (rho theta) per point (mu_ref <= 0: the constant tau)."""
        lib().oracle_set_viscosity(self.h, float(mu_ref), float(omega))

    def set_geometry(self, x):
        """Curvilinear hexahedra: physical coordinates x [n_x, 3] of every solution node."""
        x = _f64(x, (self.npts, 3))
        rc = lib().oracle_set_geometry(self.h, _d(x))
        if rc != 0:
            raise ValueError(f"oracle_set_geometry: {rc}")

    def set_connectivity(self, nbr, nface, orient):
        """Unstructured connectivity: [nelem, 6] neighbour / shared face / orientation tables."""
        a = [np.ascontiguousarray(t, dtype=np.int32).reshape(-1) for t in (nbr, nface, orient)]
        rc = lib().oracle_set_connectivity(self.h, _i(a[0]), _i(a[1]), _i(a[2]))
        if rc != 0:
            raise ValueError(f"oracle_set_connectivity: {rc}")

    def metric(self):
        """(Ja [n_x, 3, 3] with Ja[:, i, n] = J d r_i / d x_n, J [n_x]) of the curvilinear geometry."""
        Ja = np.zeros((self.npts, 3, 3))
        J = np.zeros(self.npts)
        assert lib().oracle_metric(self.h, _d(Ja), _d(J)) == 0
        return Ja, J

    def face_elements(self, fc):
        """Elements on face fc = 2 d + side (the product of the other directions' counts)."""
        ne = [max(1, int(n)) for n in self._keep[0]]
        d = fc // 2
        return int(np.prod([ne[q] for q in range(3) if q != d]))

    def stage(self, dt, stage):
        """One Shu-Osher stage (0, 1, 2) of oracle_step's RK3 step."""
        rc = lib().oracle_stage(self.h, float(dt), int(stage))
        if rc != 0:
            raise RuntimeError(f"oracle_stage: {rc}")

    def pack_halo(self, fc, stage):
        """The element layer next to face fc of the source of `stage`: [face element][node][velocity]."""
        nel = int(np.prod([max(1, int(n)) for n in self._keep[0]]))
        out = np.zeros((self.face_elements(fc), self.npts // nel, self.nvel))
        assert lib().oracle_pack_halo(self.h, int(fc), int(stage), _d(out)) == 0
        return out

    def set_halo(self, fc, halo):
        """The halo of exchange face fc, [face element][node][velocity]."""
        a = _f64(halo)
        assert lib().oracle_set_halo(self.h, int(fc), _d(a)) == 0

    def set_limiter(self, on):
        lib().oracle_set_limiter(self.h, int(bool(on)))

    def limit(self, f):
        """The positivity limiter applied to a copy of f [n_x, N_v]."""
        a = np.ascontiguousarray(f, dtype=np.float64).reshape(self.npts, self.nvel).copy()
        lib().oracle_limit(self.h, _d(a))
        return a
