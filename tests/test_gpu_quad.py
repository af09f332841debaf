"""Quadrilateral elements (dim = 2, the planar problems) on the GPU against the FP64 oracle: single
steps at p = 1-3 in the three- and two-dimensional velocity spaces with ragged element blocks and
tiles, a Dirichlet tube with the limiter in the FP32-split and all-FP64 forms, the variable collision
time, periodic conservation, and a y-independent state that must evolve as the line problem."""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_2308_06196_gb300 import _build, workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    _build.build()


def rel(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


def grid(n, L, m):
    return ((n, n, n), (-L,) * 3, (L,) * 3) if m == 3 else ((n, n, 1), (-L, -L, 0.0), (L, L, 0.0))


def make(ne, p, n=6, L=4.0, tau=0.05, m=3, bc=None, bcs=None, limiter=False, **opts):
    from paper_2308_06196_gb300.bgk import Solver

    g = grid(n, L, m)
    s = Solver(2, list(ne), (0.0, 0.0), (1.0, 1.0), p, *g, tau, bc=bc, bc_state=bcs, limiter=limiter, **opts)
    pr = orc.Problem(2, list(ne), [0.0, 0.0], [1.0, 1.0], p, *g, tau,
                     bc=None if bc is None else np.asarray(bc).reshape(6),
                     bc_state=None if bcs is None else np.asarray(bcs, dtype=float).reshape(30))
    pr.set_limiter(limiter)
    return s, pr


def prim2(x, seed, m, amp=0.2):
    P = W.smooth_prim(x, 2, seed=seed, amp=amp)
    if m == 2:
        P[:, 3] = 0.0
    return P


@pytest.mark.parametrize("p", [1, 2, 3])
@pytest.mark.parametrize("m,n", [(3, 6), (2, 10)])
@pytest.mark.parametrize("opts", [dict(), dict(chunks=1, vtiles_per_task=1)])
def test_steps_vs_oracle(p, m, n, opts):
    # 5 x 3 elements: not a multiple of the 4-element CTA block; 6^3 (octants of 27) and 10^2 (quadrants
    # of 25) velocities: padded tiles
    s, pr = make((5, 3), p, n=n, m=m, **opts)
    pr.set_state(prim2(pr.points(), 30 + p, m))
    f = pr.get_f() * W.noise((pr.npts, pr.nvel), seed=40 + p, amp=0.05)
    s.set_f(f)
    pr.set_f(f.astype(np.float32).astype(np.float64))
    dt = pr.dt(0.1)
    assert abs(s.dt(0.1) - dt) <= 1e-14 * dt
    s.step(dt, 3)
    pr.step(dt, 3)
    assert rel(s.get_f(), pr.get_f()) < 1e-5
    assert rel(s.moments(), pr.moments()) < 1e-5


def tube():
    bc = [[W.DIRICHLET, W.DIRICHLET], [0, 0], [0, 0]]
    bcs = np.zeros((3, 2, 5))
    bcs[0, 0] = [1.0, 0.0, 0.0, 0.0, 1.0]
    bcs[0, 1] = [0.2, 0.0, 0.0, 0.0, 0.8]
    return bc, bcs


@pytest.mark.parametrize("precision,tol", [(0, 1e-5), (1, 1e-10)])
@pytest.mark.parametrize("m", [2, 3])
def test_dirichlet_tube_with_limiter(precision, tol, m):
    bc, bcs = tube()
    s, pr = make((8, 2), 3, n=12 if m == 2 else 8, L=6.0, tau=1e-3, m=m, bc=bc, bcs=bcs, limiter=True,
                 precision=precision)
    prim = W.prim_sod(pr.points(), (1.0, 1.0), (0.2, 0.8))
    s.set_state(prim)
    pr.set_state(prim)
    dt = pr.dt(0.1)
    s.step(dt, 6)
    pr.step(dt, 6)
    assert rel(s.moments(), pr.moments()) < tol
    assert rel(s.get_f(), pr.get_f()) < tol


def test_variable_tau_vs_oracle():
    s, pr = make((4, 3), 2, n=10, L=5.0, tau=1.0, m=2, mu_ref=2e-3, mu_omega=0.81)
    pr.set_viscosity(2e-3, 0.81)
    prim = prim2(pr.points(), 7, 2, amp=0.3)
    s.set_state(prim)
    pr.set_state(prim)
    dt = min(pr.dt(0.1), s.dt(0.1))
    s.step(dt, 4)
    pr.step(dt, 4)
    assert rel(s.moments(), pr.moments()) < 1e-5


def test_periodic_conservation_100_steps():
    p, ne = 3, (4, 4)
    s, pr = make(ne, p, n=12, L=6.0, tau=0.01, m=2)
    s.set_state(prim2(s.points(), 9, 2, amp=0.3))
    _, w = orc.gauss_legendre(p + 1)
    Wn = np.outer(w, w).ravel()

    def tot(Q):
        return (Q.reshape(-1, Wn.size, 5) * Wn[None, :, None]).sum((0, 1))

    T0 = tot(s.moments())
    s.step(s.dt(0.1), 100)
    Q = s.moments()
    assert np.all(Q[:, 3] == 0.0)
    assert np.abs(tot(Q) - T0).max() <= 2e-6 * np.abs(T0).max()


def test_y_independent_state_is_the_line():
    from paper_2308_06196_gb300.bgk import Solver

    p, ne, n, L = 3, 6, 10, 5.0
    g = grid(n, L, 2)
    s1 = Solver(1, [ne], [0.0], [1.0], p, *g, 0.02)
    s2 = Solver(2, [ne, 3], [0.0, 0.0], [1.0, 1.0], p, *g, 0.02)

    def prim(x):
        sn = np.sin(2 * np.pi * x[:, 0])
        return np.stack([1 + 0.2 * sn, 0.1 * np.cos(2 * np.pi * x[:, 0]), 0.05 * sn, 0 * sn, 1 + 0.1 * sn], 1)

    x1, x2 = s1.points(), s2.points()
    s1.set_state(prim(x1))
    s2.set_state(prim(x2))
    dt = s1.dt(0.1)
    s1.step(dt, 10)
    s2.step(dt, 10)
    idx = np.array([np.argmin(np.abs(x1[:, 0] - xx)) for xx in x2[:, 0]])
    assert rel(s2.moments(), s1.moments()[idx]) < 2e-6


def test_dirichlet_in_y_vs_oracle():
    # the other face pair: Dirichlet data at y = 0 and y = 1, periodic in x
    bc = [[0, 0], [W.DIRICHLET, W.DIRICHLET], [0, 0]]
    bcs = np.zeros((3, 2, 5))
    bcs[1, 0] = [1.0, 0.1, 0.0, 0.0, 1.0]
    bcs[1, 1] = [0.4, 0.0, -0.1, 0.0, 0.9]
    s, pr = make((3, 5), 2, n=8, L=5.0, tau=0.01, m=3, bc=bc, bcs=bcs)
    prim = prim2(pr.points(), 11, 3)
    s.set_state(prim)
    pr.set_state(prim)
    dt = pr.dt(0.1)
    s.step(dt, 4)
    pr.step(dt, 4)
    assert rel(s.moments(), pr.moments()) < 1e-5
    assert rel(s.get_f(), pr.get_f()) < 1e-5
