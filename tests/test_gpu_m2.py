"""The two-dimensional velocity space (velocity dimension m = 2: the third grid axis has one node) on
the GPU against the FP64 oracle: the Newton solve's moments, single steps and a Dirichlet tube on
line elements in the FP32-split and all-FP64 forms, periodic conservation, the exact relaxation of a
uniform state, a batch of m = 2 members, and the allocation-free entry point."""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_2308_06196_gb300 import _build, workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    _build.build()


def make(ne, p, n, L=6.0, tau=0.05, bc=None, bcs=None, **opts):
    from paper_2308_06196_gb300.bgk import Solver

    grid = ((n, n, 1), (-L, -L, 0.0), (L, L, 0.0))
    s = Solver(1, [ne], [0.0], [1.0], p, *grid, tau, bc=bc, bc_state=bcs, **opts)
    pr = orc.Problem(1, [ne], [0.0], [1.0], p, *grid, tau,
                     bc=None if bc is None else np.asarray(bc).reshape(6),
                     bc_state=None if bcs is None else np.asarray(bcs, dtype=float).reshape(30))
    return s, pr


def psi2(xi):
    return np.stack([np.ones(len(xi)), xi[:, 0], xi[:, 1], np.zeros(len(xi)), 0.5 * (xi[:, :2] ** 2).sum(1)], 1)


def maxwell2(xi, P):
    return P[0] / (2 * np.pi * P[4]) * np.exp(-((xi[:, :2] - P[1:3]) ** 2).sum(1) / (2 * P[4]))


def planar_prim(x, seed, amp=0.2):
    P = W.smooth_prim(x, 1, seed=seed, amp=amp)
    P[:, 3] = 0.0
    return P


def rel(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


@pytest.mark.parametrize("n", [8, 12])
def test_newton_matches_moments(n):
    s, pr = make(3, 2, n)
    pr.set_state(planar_prim(pr.points(), 3))
    f = pr.get_f() * W.noise((pr.npts, pr.nvel), seed=4, amp=0.2)
    s.set_f(f)
    Q, P = s.moments(), s.equilibrium()
    assert np.all(Q[:, 3] == 0.0) and np.all(P[:, 3] == 0.0)
    for q, pp in zip(Q, P):
        Qg = (pr.w * maxwell2(pr.xi, pp)) @ psi2(pr.xi)
        assert np.all(np.abs(Qg - q) <= 1e-12 * np.abs(q).max())
    assert rel(Q, pr.moments(f.astype(np.float32).astype(np.float64))) < 2e-7
    Po, _, _, bad = pr.conservative_maxwellian(Q)
    assert bad == 0
    assert np.allclose(P, Po, rtol=1e-10, atol=1e-12)


@pytest.mark.parametrize("p", [1, 2, 3])
@pytest.mark.parametrize("opts", [dict(), dict(chunks=1), dict(vtiles_per_task=1)])
def test_steps_vs_oracle(p, opts):
    # 10^2 velocities: quadrants of 25 (ragged 32-velocity tiles); 5 elements (a ragged CTA block)
    s, pr = make(5, p, 10, L=5.0, tau=0.02, **opts)
    pr.set_state(planar_prim(pr.points(), 20 + p))
    f = pr.get_f() * W.noise((pr.npts, pr.nvel), seed=30 + p, amp=0.05)
    s.set_f(f)
    pr.set_f(f.astype(np.float32).astype(np.float64))
    dt = pr.dt(0.1)
    assert abs(s.dt(0.1) - dt) < 1e-15
    s.step(dt, 3)
    pr.step(dt, 3)
    assert rel(s.get_f(), pr.get_f()) < 1e-5
    assert rel(s.moments(), pr.moments()) < 1e-5


@pytest.mark.parametrize("precision,tol", [(0, 1e-5), (1, 1e-10)])
def test_dirichlet_tube_vs_oracle(precision, tol):
    bc = [[W.DIRICHLET, W.DIRICHLET], [0, 0], [0, 0]]
    bcs = np.zeros((3, 2, 5))
    bcs[0, 0] = [1.0, 0.0, 0.0, 0.0, 1.0]
    bcs[0, 1] = [0.25, 0.0, 0.0, 0.0, 0.8]
    s, pr = make(10, 3, 16, L=7.0, tau=2e-3, bc=bc, bcs=bcs, precision=precision)
    prim = W.prim_sod(pr.points(), (1.0, 1.0), (0.25, 0.8))
    s.set_state(prim)
    pr.set_state(prim)
    dt = pr.dt(0.1)
    s.step(dt, 10)
    pr.step(dt, 10)
    assert rel(s.moments(), pr.moments()) < tol
    assert rel(s.get_f(), pr.get_f()) < tol


def test_periodic_conservation_100_steps():
    p, ne = 3, 8
    s, pr = make(ne, p, 12, L=6.0, tau=0.01)
    s.set_state(planar_prim(s.points(), 5, amp=0.3))
    _, w = orc.gauss_legendre(p + 1)

    def tot(Q):
        return (Q.reshape(ne, p + 1, 5) * w[None, :, None]).sum((0, 1))

    T0 = tot(s.moments())
    s.step(s.dt(0.1), 100)
    Q = s.moments()
    assert np.all(Q[:, 3] == 0.0)
    assert np.abs(tot(Q) - T0).max() <= 2e-6 * np.abs(T0).max()


def test_space_homogeneous_relaxation():
    tau = 0.01
    s, pr = make(2, 1, 12, tau=tau)
    f0 = maxwell2(pr.xi, np.array([1.0, 0.4, -0.3, 0.0, 0.8])) + maxwell2(pr.xi, np.array([0.3, -0.8, 0.5, 0.0, 0.5]))
    F0 = np.tile(f0, (pr.npts, 1))
    s.set_f(F0)
    f0 = F0[0].astype(np.float32).astype(np.float64)
    P = pr.conservative_maxwellian(((pr.w * f0) @ psi2(pr.xi))[None])[0][0]
    M = maxwell2(pr.xi, P)
    dt, n = 0.2 * tau, 25
    s.step(dt, n)
    z = -dt / tau
    R = 1 + z + z * z / 2 + z**3 / 6
    assert np.abs(s.get_f() - (M + (f0 - M) * R**n)).max() <= 5e-6 * f0.max()


def test_batch_of_planar_members_equals_members_alone():
    from paper_2308_06196_gb300.bgk import Batch

    shapes = [(6, 2, 12), (9, 3, 16), (4, 3, 8), (13, 2, 10)]

    def build():
        out = []
        for q, (ne, p, n) in enumerate(shapes):
            s, _ = make(ne, p, n, tau=0.02 * (q + 1), chunks=1)
            s.set_state(planar_prim(s.points(), 40 + q))
            out.append(s)
        return out

    alone, batched = build(), build()
    dts = [x.dt(0.1) for x in alone]
    for x, dt in zip(alone, dts):
        x.step(dt, 5)
    b = Batch(batched)
    b.step(dts, 5)
    b.synchronize()
    for q, (xa, xb) in enumerate(zip(alone, batched)):
        assert rel(xb.moments(), xa.moments()) <= 1e-6, q
    b.close()


def test_planar_velocity_space_needs_dim_at_most_2():
    from paper_2308_06196_gb300.bgk import BGK_EINVAL, BgkError, Solver

    with pytest.raises(BgkError) as err:
        Solver(3, [2, 2, 2], [0.0] * 3, [1.0] * 3, 2, (8, 8, 1), (-4.0, -4.0, 0.0), (4.0, 4.0, 0.0), 0.1)
    assert err.value.code == BGK_EINVAL
