"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle, element by element, on
seeded inputs; plus properties checked at the full Taylor-Green size.

Tolerances (FP32-split form). f is stored in FP32 (unit round-off 6e-8) and one stage does O(50)
FP32 operations per value on O(1) data, the BGK Maxwellian is evaluated by exp2 of an FP32
exponent (relative error ~1e-6 for exponents of magnitude ~10), so one step differs from the
FP64 oracle by a few 1e-6 of max|f|; moments are sums with positive weights and carry the same
relative error. The method's own tolerance for the split form is 1e-5 relative in the moments
after 100 steps. The Newton solve is FP64 and is checked to 1e-12 on its own inputs.
"""
import math

import numpy as np
import pytest

from oracle import oracle as orc
from paper_2308_06196_gb300 import _build, workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    _build.build()


def solver(c, **opts):
    from paper_2308_06196_gb300.bgk import Solver

    k = W.mesh_kwargs(c)
    if c.get("force") is not None:
        opts.setdefault("body_force", c["force"])
    return Solver(k["dim"], k["nelem"], k["lo"], k["hi"], k["p"], k["nv"], k["vlo"], k["vhi"], k["tau"],
                  bc=c.get("bc"), bc_state=c.get("bc_state"), **opts)


def oracle_problem(c):
    k = W.mesh_kwargs(c)
    bc = c.get("bc")
    bcs = c.get("bc_state")
    return orc.Problem(k["dim"], k["nelem"], k["lo"], k["hi"], k["p"], k["nv"], k["vlo"], k["vhi"], k["tau"],
                       bc=None if bc is None else np.asarray(bc).reshape(6),
                       bc_state=None if bcs is None else np.asarray(bcs, dtype=float).reshape(30),
                       force=c.get("force"))


def psi(xi):
    return np.stack([np.ones(len(xi)), xi[:, 0], xi[:, 1], xi[:, 2], 0.5 * (xi**2).sum(1)], 1)


def maxwell(xi, P):
    return P[0] / (2 * np.pi * P[4]) ** 1.5 * np.exp(-((xi - P[1:4]) ** 2).sum(1) / (2 * P[4]))


def random_f(pr, seed, amp=0.05):
    """A seeded smooth state: the oracle's sampled Maxwellian of a smooth field, perturbed."""
    pr.set_state(W.smooth_prim(pr.points(), pr.dim, seed=seed))
    return pr.get_f() * W.noise((pr.npts, pr.nvel), seed=seed + 1, amp=amp)


def small(dim, ne, p, n, L=5.0, tau=0.05, **kw):
    c = dict(dim=dim, nelem=tuple(ne), lo=(0.0,) * dim, hi=(1.0,) * dim, p=p, nv=(n, n, n), vlo=(-L,) * 3,
             vhi=(L,) * 3, tau=tau)
    c.update(kw)
    return c


def rel(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


# ------------------------------------------------------------------------------------------------


@pytest.mark.parametrize("n", [6, 10])
def test_newton_matches_moments(n):
    c = small(1, [3], 2, n)
    pr = oracle_problem(c)
    f = random_f(pr, seed=3, amp=0.2)
    s = solver(c)
    s.set_f(f)
    Q = s.moments()
    P = s.equilibrium()
    # FP64 Newton: discrete moments of the returned Maxwellian equal the library's moments
    for q, pp in zip(Q, P):
        Qg = (pr.w * maxwell(pr.xi, pp)) @ psi(pr.xi)
        assert np.all(np.abs(Qg - q) <= 1e-12 * np.abs(q).max())
    # the moments are those of the FP32-stored f (exact double-float sums of FP32 partials)
    f32 = f.astype(np.float32).astype(np.float64)
    Qo = pr.moments(f32)
    assert rel(Q, Qo) < 2e-7
    # and the equilibrium is the oracle's (unique) solution for the same moments
    Po, it, res, bad = pr.conservative_maxwellian(Q)
    assert bad == 0
    assert np.allclose(P, Po, rtol=1e-10, atol=1e-12)


@pytest.mark.parametrize("p", [1, 2, 3])
@pytest.mark.parametrize("opts", [dict(), dict(chunks=1, vtiles_per_task=1), dict(vtiles_per_task=3)])
def test_one_step_3d(p, opts):
    # 3 x 2 x 3 elements (not a multiple of the 4 elements per CTA), 6^3 and 10^3 grids (octants of
    # 27 and 125 velocities: ragged 32-velocity tiles)
    for n in (6, 10):
        c = small(3, [3, 2, 3], p, n, L=4.0, tau=0.05)
        pr = oracle_problem(c)
        f = random_f(pr, seed=10 + p)
        s = solver(c, **opts)
        s.set_f(f)
        pr.set_f(f.astype(np.float32).astype(np.float64))
        dt = pr.dt(0.1)
        assert abs(s.dt(0.1) - dt) < 1e-15
        s.step(dt, 1)
        pr.step(dt, 1)
        fg, fo = s.get_f(), pr.get_f()
        assert rel(fg, fo) < 5e-6, (n, rel(fg, fo))
        assert rel(s.moments(), pr.moments()) < 5e-6


@pytest.mark.parametrize("p", [1, 2, 3, 5])
def test_one_step_1d(p):
    c = small(1, [5], p, 8, L=4.0, tau=0.02)
    pr = oracle_problem(c)
    f = random_f(pr, seed=20 + p)
    s = solver(c)
    s.set_f(f)
    pr.set_f(f.astype(np.float32).astype(np.float64))
    dt = pr.dt(0.1)
    s.step(dt, 3)
    pr.step(dt, 3)
    assert rel(s.get_f(), pr.get_f()) < 1e-5
    assert rel(s.moments(), pr.moments()) < 1e-5


def test_periodic1d_100_steps_moments():
    # the 1-D correctness workload at full size: moments within 1e-5 relative after 100 steps
    c = W.config("periodic1d")
    pr = oracle_problem(c)
    s = solver(c)
    prim = W.prim_field("periodic1d", pr.points())
    pr.set_state(prim)
    s.set_state(prim)
    dt = pr.dt(c["cfl"])
    s.step(dt, c["steps"])
    pr.step(dt, c["steps"])
    Qg, Qo = s.moments(), pr.moments()
    for comp in (0, 4):
        assert np.abs(Qg[:, comp] - Qo[:, comp]).max() <= 1e-5 * np.abs(Qo[:, comp]).max()
    assert np.abs(Qg[:, 1:4] - Qo[:, 1:4]).max() <= 1e-5 * np.abs(Qo[:, 0]).max()


def test_free_stream_gpu():
    # a state constant in space (a perturbed Maxwellian in velocity): advection leaves it unchanged
    # and a negligible relaxation (tau = 1e30) leaves only the round-off of the RK coefficients
    c = small(3, [2, 3, 2], 3, 6, tau=1e30)
    s = solver(c)
    pr = oracle_problem(c)
    rng = np.random.default_rng(4)
    f = np.tile(pr.sample_maxwellian([1.0, 0.2, -0.1, 0.3, 1.1]) * rng.uniform(0.9, 1.1, 216), (s.npts, 1))
    s.set_f(f)
    s.step(0.001, 10)
    f32 = f.astype(np.float32).astype(np.float64)
    assert rel(s.get_f(), f32) < 10 * 2 * 6e-8


def test_space_homogeneous_relaxation_gpu():
    tau = 0.01
    c = small(1, [2], 1, 10, tau=tau)
    pr = oracle_problem(c)
    rng = np.random.default_rng(9)
    xi = pr.xi
    f0 = maxwell(xi, np.array([1.0, 0.3, -0.2, 0.1, 0.8])) + maxwell(xi, np.array([0.4, -0.5, 0.4, 0.0, 0.5]))
    f0 *= 1 + 0.01 * rng.uniform(-1, 1, len(f0))
    F0 = np.tile(f0, (pr.npts, 1))
    s = solver(c)
    s.set_f(F0)
    f0 = F0[0].astype(np.float32).astype(np.float64)
    Q = (pr.w * f0) @ psi(xi)
    P = pr.conservative_maxwellian(Q[None])[0][0]
    M = maxwell(xi, P)
    dt, n = 0.2 * tau, 25
    s.step(dt, n)
    z = -dt / tau
    R = 1 + z + z * z / 2 + z**3 / 6
    exact = M + (f0 - M) * R**n
    assert np.abs(s.get_f() - exact).max() <= 5e-6 * f0.max()


def test_conservation_gpu_periodic():
    c = small(3, [2, 2, 2], 2, 8, L=4.0, tau=0.02)
    s = solver(c)
    x = s.points()
    s.set_state(W.smooth_prim(x, 3, seed=5))
    _, Wg = orc.gauss_legendre(3)
    Wn = np.einsum("i,j,k->kji", Wg, Wg, Wg).ravel()

    def glob(Q):  # spatial integral up to the constant element Jacobian
        return (Q.reshape(-1, 27, 5) * Wn[None, :, None]).sum((0, 1))

    G0 = glob(s.moments())
    s.step(s.dt(0.1), 100)
    G1 = glob(s.moments())
    # FP32 storage: round-off level drift, relative to the mass and energy scale
    assert np.abs(G1 - G0).max() <= 2e-6 * max(abs(G0[0]), abs(G0[4]))


def test_dirichlet_ends_1d():
    # Sod-like tube with Dirichlet Maxwellian ends
    left, right = [1.0, 0, 0, 0, 1.0], [0.3, 0, 0, 0, 0.8]
    bc = [[W.DIRICHLET, W.DIRICHLET], [0, 0], [0, 0]]
    bcs = np.zeros((3, 2, 5))
    bcs[0, 0], bcs[0, 1] = left, right
    c = small(1, [8], 2, 8, L=4.0, tau=0.01, bc=bc, bc_state=bcs)
    pr = oracle_problem(c)
    x = pr.points()[:, 0]
    prim = np.where((x < 0.5)[:, None], np.array(left)[None], np.array(right)[None])
    pr.set_state(prim)
    s = solver(c)
    s.set_state(prim)
    dt = pr.dt(0.1)
    s.step(dt, 10)
    pr.step(dt, 10)
    assert rel(s.moments(), pr.moments()) < 1e-5
    assert rel(s.get_f(), pr.get_f()) < 1e-5


def test_taylor_green_reduced_mesh_full_velocity_grid():
    # the Taylor-Green workload's kernel configuration (p = 3 hexahedra, 24^3 velocities, 8 octant
    # chunks) on a 4^3-element mesh the oracle can step in seconds
    c = W.config("taylor_green", nelem=(4, 4, 4))
    pr = oracle_problem(c)
    s = solver(c)
    prim = W.prim_field("taylor_green", pr.points())
    pr.set_state(prim)
    s.set_state(prim)
    dt = pr.dt(c["cfl"])
    s.step(dt, 1)
    pr.step(dt, 1)
    Qg, Qo = s.moments(), pr.moments()
    assert np.abs(Qg - Qo).max() <= 1e-5 * np.abs(Qo[:, [0, 4]]).max()
    assert rel(s.get_f(), pr.get_f()) < 1e-5


def test_taylor_green_full_size_properties():
    # full size (16^3 hexahedra at p = 3, 24^3 velocities, 3.6e9 DOF), the benchmarked configuration:
    # conservation of the global moments, the Newton solution at sampled points, determinism
    c = W.config("taylor_green")
    s = solver(c)
    x = s.points()
    prim = W.prim_field("taylor_green", x)
    s.set_state(prim)
    Q0 = s.moments()
    dt = s.dt(c["cfl"])
    s.step(dt, 2)
    Q1 = s.moments()
    P1 = s.equilibrium()
    _, Wg = orc.gauss_legendre(4)
    Wn = np.einsum("i,j,k->kji", Wg, Wg, Wg).ravel()
    G0 = (Q0.reshape(-1, 64, 5) * Wn[None, :, None]).sum((0, 1))
    G1 = (Q1.reshape(-1, 64, 5) * Wn[None, :, None]).sum((0, 1))
    assert np.abs(G1 - G0).max() <= 1e-6 * max(G0[0], G0[4])
    xi, w = orc.velocity_grid(c["nv"], c["vlo"], c["vhi"])
    rng = np.random.default_rng(0)
    for pt in rng.choice(len(Q1), 32, replace=False):
        Qg = (w * maxwell(xi, P1[pt])) @ psi(xi)
        assert np.all(np.abs(Qg - Q1[pt]) <= 1e-12 * np.abs(Q1[pt]).max())
    s.set_state(prim)
    s.step(dt, 2)
    assert np.array_equal(s.moments(), Q1)


# ---------------------------------------------------------------------------------------------
# the plain all-FP64 form (precision = BGK_FP64): the same method in FP64, unfused


@pytest.mark.parametrize("p", [1, 2, 3])
def test_fp64_one_step_3d(p):
    from paper_2308_06196_gb300.bgk import FP64

    c = small(3, [3, 2, 3], p, 6, L=4.0, tau=0.05)
    pr = oracle_problem(c)
    f = random_f(pr, seed=40 + p)
    s = solver(c, precision=FP64)
    s.set_f(f)
    pr.set_f(f)
    dt = pr.dt(0.1)
    s.step(dt, 2)
    pr.step(dt, 2)
    # FP64 on both sides: differences come from summation order and the two Newton solvers
    # (each converged to ~1e-13 of the moments)
    assert rel(s.get_f(), pr.get_f()) < 1e-10
    assert rel(s.moments(), pr.moments()) < 1e-10


def test_fp64_periodic1d_100_steps_and_conservation():
    from paper_2308_06196_gb300.bgk import FP64

    c = W.config("periodic1d")
    pr = oracle_problem(c)
    s = solver(c, precision=FP64)
    prim = W.prim_field("periodic1d", pr.points())
    pr.set_state(prim)
    s.set_state(prim)
    Q0 = s.moments()
    dt = pr.dt(c["cfl"])
    s.step(dt, c["steps"])
    pr.step(dt, c["steps"])
    Qg, Qo = s.moments(), pr.moments()
    assert np.abs(Qg - Qo).max() <= 1e-10 * np.abs(Qo).max()
    _, Wg = orc.gauss_legendre(4)
    G0 = (Q0.reshape(-1, 4, 5) * Wg[None, :, None]).sum((0, 1))
    G1 = (Qg.reshape(-1, 4, 5) * Wg[None, :, None]).sum((0, 1))
    assert np.abs(G1 - G0).max() <= 1e-12 * max(abs(G0[0]), abs(G0[4]))


def test_fp64_free_stream():
    from paper_2308_06196_gb300.bgk import FP64

    c = small(3, [2, 3, 2], 3, 6, tau=1e30)
    s = solver(c, precision=FP64)
    pr = oracle_problem(c)
    rng = np.random.default_rng(4)
    f = np.tile(pr.sample_maxwellian([1.0, 0.2, -0.1, 0.3, 1.1]) * rng.uniform(0.9, 1.1, 216), (s.npts, 1))
    s.set_f(f)
    s.step(0.001, 10)
    assert rel(s.get_f(), f) < 1e-13


# ---------------------------------------------------------------------------------------------
# diffuse walls and the body force (the channel workload's boundary and source)


def small_channel(**kw):
    return W.config("channel", nelem=(4, 3, 2), hi=(1.0, 1.0, 0.5), nv=(8, 8, 8), vlo=(-5.0,) * 3,
                    vhi=(5.0,) * 3, **kw)


@pytest.mark.parametrize("fp64", [False, True])
def test_channel_walls_and_force_vs_oracle(fp64):
    from paper_2308_06196_gb300.bgk import FP64, FP32_SPLIT

    c = small_channel(force=(0.05, 0.02, 0.0))
    pr = oracle_problem(c)
    s = solver(c, precision=FP64 if fp64 else FP32_SPLIT)
    # a non-uniform state so the walls see different densities at every face point
    f = random_f(pr, seed=50)
    s.set_f(f)
    pr.set_f(f if fp64 else f.astype(np.float32).astype(np.float64))
    dt = pr.dt(0.1)
    s.step(dt, 3)
    pr.step(dt, 3)
    tol = 1e-10 if fp64 else 1e-5
    assert rel(s.get_f(), pr.get_f()) < tol
    assert rel(s.moments(), pr.moments()) < tol


@pytest.mark.parametrize("fp64", [False, True])
def test_channel_mass_conserved_momentum_driven(fp64):
    # walls have zero net discrete mass flux and x, z are periodic: total mass is conserved; at rest
    # the first step gains x-momentum rho F dt per unit volume (no wall shear yet)
    from paper_2308_06196_gb300.bgk import FP64, FP32_SPLIT

    c = small_channel()
    s = solver(c, precision=FP64 if fp64 else FP32_SPLIT)
    s.set_state(W.prim_field("channel", s.points()))
    _, Wg = orc.gauss_legendre(3)
    Wn = np.einsum("i,j,k->kji", Wg, Wg, Wg).ravel()
    vol = 1.0 * 1.0 * 0.5
    jac = vol / (4 * 3 * 2) / 8.0  # element volume / reference volume

    def glob(Q):
        return (Q.reshape(-1, 27, 5) * Wn[None, :, None]).sum((0, 1)) * jac

    G0 = glob(s.moments())
    dt = s.dt(0.1)
    s.step(dt, 1)
    G1 = glob(s.moments())
    assert abs(G1[1] - G0[1] - G0[0] * 0.01 * dt) <= 0.05 * G0[0] * 0.01 * dt
    s.step(dt, 19)
    G2 = glob(s.moments())
    assert abs(G2[0] - G0[0]) <= (1e-12 if fp64 else 2e-6) * G0[0]


@pytest.mark.parametrize("fp64", [False, True])
def test_general_form_reruns_are_bit_identical(fp64):
    # walls (their densities summed over 4 warps in a fixed order), body force, limiter and variable tau:
    # two fresh contexts on the same input give the same f and moments, bit for bit
    from paper_2308_06196_gb300.bgk import FP64, FP32_SPLIT

    c = small_channel(force=(0.05, 0.02, 0.0))
    f = random_f(oracle_problem(c), seed=51)
    runs = []
    for _ in range(2):
        s = solver(c, precision=FP64 if fp64 else FP32_SPLIT, limiter=True, mu_ref=2e-2, mu_omega=0.81)
        s.set_f(f)
        dt = s.dt(0.1)
        s.step(dt, 3)
        runs.append((s.get_f(), s.moments()))
        s.close()
    assert np.array_equal(runs[0][0], runs[1][0])
    assert np.array_equal(runs[0][1], runs[1][1])


def test_autotune_keeps_results():
    # the autotuner only changes the task shape: the same step gives the same moments (the grouping of
    # the FP32 partial sums changes, so agreement is to FP32 summation order, not bitwise)
    c = small(3, [3, 2, 3], 3, 10, L=4.0, tau=0.05)
    pr = oracle_problem(c)
    f = random_f(pr, seed=60)
    a = solver(c)
    b = solver(c)
    G = b.autotune()
    assert G in (2, 4, 8, 16)
    a.set_f(f)
    b.set_f(f)
    dt = pr.dt(0.1)
    a.step(dt, 2)
    b.step(dt, 2)
    assert rel(a.moments(), b.moments()) < 1e-6
    assert rel(a.get_f(), b.get_f()) < 1e-6
