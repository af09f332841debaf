"""Edge cases of the GPU path against the FP64 oracle: velocity grids with a different spacing, node
count and extent on every axis (asymmetric about 0), in both precisions, in 3-D and 1-D; meshes of a
single element per direction (periodic: every element is its own upwind neighbour); the smallest
velocity grid with a unique conservative Maxwellian (3 nodes per axis, the centre node joining the
positive octant); and the velocity grid whose energy moment depends on the others (2 nodes on every
axis), rejected before anything is allocated."""
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


def pair(dim, ne, p, nv, vlo, vhi, tau, **opts):
    from paper_2308_06196_gb300.bgk import Solver

    lo, hi = [0.0] * dim, [1.0] * dim
    s = Solver(dim, list(ne), lo, hi, p, nv, vlo, vhi, tau, **opts)
    pr = orc.Problem(dim, list(ne), lo, hi, p, nv, vlo, vhi, tau)
    return s, pr


def run_both(s, pr, seed, steps, precision=0, amp=0.05):
    pr.set_state(W.smooth_prim(pr.points(), pr.dim, seed=seed, amp=0.2))
    f = pr.get_f() * W.noise((pr.npts, pr.nvel), seed=seed + 1, amp=amp)
    s.set_f(f)
    pr.set_f(f if precision == 1 else f.astype(np.float32).astype(np.float64))
    dt = pr.dt(0.1)
    assert abs(s.dt(0.1) - dt) <= 1e-13 * dt
    s.step(dt, steps)
    pr.step(dt, steps)


ANISO = dict(nv=(6, 8, 10), vlo=(-4.0, -5.0, -3.5), vhi=(4.5, 5.0, 3.0))


@pytest.mark.parametrize("precision,tol", [(0, 1e-5), (1, 1e-10)])
@pytest.mark.parametrize("dim,ne,p", [(3, (3, 2, 2), 2), (1, (6,), 3)])
def test_anisotropic_asymmetric_velocity_grid_vs_oracle(precision, tol, dim, ne, p):
    # per-axis spacings select the general stage kernel (per-axis exponent terms and moment weights)
    s, pr = pair(dim, ne, p, ANISO["nv"], ANISO["vlo"], ANISO["vhi"], 0.05, precision=precision)
    run_both(s, pr, seed=70 + dim, steps=3, precision=precision)
    assert rel(s.moments(), pr.moments()) < tol
    assert rel(s.get_f(), pr.get_f()) < tol


@pytest.mark.parametrize("precision,tol", [(0, 1e-5), (1, 1e-10)])
@pytest.mark.parametrize("dim,ne,p", [(3, (1, 1, 1), 3), (3, (1, 2, 3), 2), (1, (1,), 3)])
def test_single_element_directions_vs_oracle(precision, tol, dim, ne, p):
    s, pr = pair(dim, ne, p, (6, 6, 6), (-4.0,) * 3, (4.0,) * 3, 0.05, precision=precision)
    run_both(s, pr, seed=80 + p, steps=3, precision=precision)
    assert rel(s.moments(), pr.moments()) < tol
    assert rel(s.get_f(), pr.get_f()) < tol


def test_three_nodes_per_axis_vs_oracle():
    # octants of 8, 4, 2 and 1 velocities (the centre node joins the positive side): tiles almost all
    # padding
    s, pr = pair(3, (2, 2, 2), 2, (3, 3, 3), (-2.0,) * 3, (2.0,) * 3, 0.05)
    run_both(s, pr, seed=90, steps=3, amp=0.02)
    assert rel(s.moments(), pr.moments()) < 1e-5
    assert rel(s.get_f(), pr.get_f()) < 1e-5


@pytest.mark.parametrize("nv", [(2, 2, 2), (2, 2, 1)])
def test_two_nodes_on_every_axis_rejected(nv):
    from paper_2308_06196_gb300.bgk import BGK_EINVAL, BgkError, Solver

    dim = 3 if nv[2] > 1 else 1
    with pytest.raises(BgkError) as err:
        Solver(dim, [2] * dim, [0.0] * dim, [1.0] * dim, 2, nv, (-4.0, -3.0, -2.0), (4.0, 5.0, 2.0), 0.05)
    assert err.value.code == BGK_EINVAL
