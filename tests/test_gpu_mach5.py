"""The Mach-5 shock duct: Rankine-Hugoniot states, Dirichlet x-ends, periodic y and z.

- a reduced duct (8 x 1 x 1 hexahedra, 24^3 velocities) against the FP64 oracle, with and without
  the positivity limiter;
- the full workload (128 x 8 x 8 hexahedra at p = 2, 48^3 velocities on [-14, 14]^3, about 2.4e10
  degrees of freedom, positivity limiter on) in the FP32-split form: the flow must stay exactly
  y/z-homogeneous (the y and z derivatives of a y/z-constant field vanish in the difference form),
  and it must match the plain all-FP64 form run on the one-element-wide duct of the same x-mesh
  within 1e-5 in the moments;
- without the limiter the duct's p = 2 solution undershoots at the shock until a point's moments
  admit no Maxwellian: the library reports it (BGK_ENEWTON / BGK_EDOMAIN) instead of going on."""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_2308_06196_gb300 import _build, workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    _build.build()


def solver(c, **opts):
    from paper_2308_06196_gb300.bgk import Solver

    k = W.mesh_kwargs(c)
    bc, bcs = W.mach5_bc(c)
    return Solver(k["dim"], k["nelem"], k["lo"], k["hi"], k["p"], k["nv"], k["vlo"], k["vhi"], k["tau"],
                  bc=bc, bc_state=bcs, **opts)


def rel(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


@pytest.mark.parametrize("limiter", [False, True])
def test_reduced_duct_vs_oracle(limiter):
    c = W.config("mach5", nelem=(8, 1, 1), hi=(16.0, 2.0, 2.0), nv=(24, 24, 24))
    k = W.mesh_kwargs(c)
    bc, bcs = W.mach5_bc(c)
    pr = orc.Problem(3, k["nelem"], k["lo"], k["hi"], k["p"], k["nv"], k["vlo"], k["vhi"], k["tau"],
                     bc=np.asarray(bc).reshape(6), bc_state=np.asarray(bcs, dtype=float).reshape(30))
    pr.set_limiter(limiter)
    s = solver(c, limiter=limiter)
    prim = W.prim_mach5(pr.points(), c)
    pr.set_state(prim)
    s.set_state(prim)
    dt = pr.dt(0.1)
    pr.step(dt, 5)
    s.step(dt, 5)
    assert rel(s.moments(), pr.moments()) < 1e-5
    assert rel(s.get_f(), pr.get_f()) < 1e-5


def test_full_duct_homogeneous_and_matches_fp64_narrow_duct():
    from paper_2308_06196_gb300.bgk import FP64

    c = W.config("mach5")
    steps = 20
    s = solver(c, limiter=c["limiter"])
    x = s.points()
    s.set_state(W.prim_mach5(x, c))
    dt = s.dt(c["cfl"])
    s.step(dt, steps)
    Q = s.moments()
    del s
    ne = c["nelem"]
    # points: element-major (x fastest), nodes x fastest: regroup by (x element, x node)
    n1 = c["p"] + 1
    Qe = Q.reshape(ne[2], ne[1], ne[0], n1, n1, n1, 5)          # ez, ey, ex, iz, iy, ix, c
    Qx = Qe.transpose(2, 5, 0, 1, 3, 4, 6).reshape(ne[0], n1, -1, 5)  # ex, ix, (ez ey iz iy), c
    assert np.array_equal(Qx, np.broadcast_to(Qx[:, :, :1], Qx.shape)), "y/z homogeneity lost"

    # the same x-mesh, one element (of the same width) in y and z, in the plain all-FP64 form
    hy = (c["hi"][1] - c["lo"][1]) / ne[1]
    c64 = dict(c, nelem=(ne[0], 1, 1), hi=(c["hi"][0], hy, hy))
    s64 = solver(c64, precision=FP64, limiter=c["limiter"])
    s64.set_state(W.prim_mach5(s64.points(), c64))
    assert abs(s64.dt(c["cfl"]) - dt) <= 1e-15 * dt
    s64.step(dt, steps)
    Q64 = s64.moments().reshape(ne[0], n1, n1, n1, 5)[:, 0, 0, :, :]  # ex, ix (iz = iy = 0), c
    rho = Q64[..., 0]
    th = (2.0 / 3.0) * (Q64[..., 4] / rho - 0.5 * (Q64[..., 1:4] ** 2).sum(-1) / rho**2)
    scale = np.array([rho.max()] + [(rho * np.sqrt(th)).max()] * 3 + [Q64[..., 4].max()])
    err = (np.abs(Qx[:, :, 0, :] - Q64) / scale).max()
    assert err <= 1e-5, err


def test_narrow_duct_without_limiter_is_reported():
    from paper_2308_06196_gb300.bgk import BgkError, BGK_EDOMAIN, BGK_ENEWTON

    c = W.config("mach5")
    c1 = dict(c, nelem=(128, 1, 1), hi=(16.0, 0.125, 0.125))
    s = solver(c1, limiter=False)
    s.set_state(W.prim_mach5(s.points(), c1))
    dt = s.dt(c["cfl"])
    with pytest.raises(BgkError) as err:
        for _ in range(20):
            s.step(dt, 1)
            s.synchronize()
    assert err.value.code in (BGK_EDOMAIN, BGK_ENEWTON)
