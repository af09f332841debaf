"""Pins of the oracle's FR advection residual (paper Sec. 2.1, Eqs. 7-9) against closed forms,
textbook schemes and an independently written weak-form DG. CPU only."""
import numpy as np
import pytest
from numpy.polynomial import legendre as npleg
from numpy.polynomial import polynomial as nppoly

from oracle import oracle as orc

INF = float("inf")


def make(dim, ne, p, nv=(2, 2, 2), vl=1.0, tau=INF, lo=None, hi=None, bc=None, bc_state=None):
    lo = lo or [0.0] * dim
    hi = hi or [1.0] * dim
    return orc.Problem(dim, list(ne), lo, hi, p, nv, (-vl,) * 3, (vl,) * 3, tau, bc=bc, bc_state=bc_state)


@pytest.mark.parametrize("dim,p", [(1, 1), (1, 3), (1, 5), (2, 2), (2, 3), (3, 1), (3, 2), (3, 3)])
def test_free_stream_preserved(dim, p):
    ne = [5] if dim == 1 else [3, 2, 2]
    pr = make(dim, ne, p, nv=(4, 3, 5), vl=5.0)
    rng = np.random.default_rng(1)
    f = np.tile(rng.uniform(0.1, 2.0, pr.nvel), (pr.npts, 1))  # constant in space per velocity
    R = pr.residual(f)
    scale = np.abs(f).max() * 5.0 * 3 * max(ne) * 2 * (p + 1) ** 2
    assert np.abs(R).max() <= 1e-13 * scale


@pytest.mark.parametrize("dim", [1, 3])
def test_p0_is_first_order_upwind(dim):
    # p = 0: one node per element, D = 0, g_L'(x0) = -1/2, so FR reduces to the textbook upwind
    # finite-volume difference -a (f_i - f_{i-1}) / h for a > 0 (mirror for a < 0), per direction.
    ne = [7] if dim == 1 else [4, 3, 5]
    pr = make(dim, ne, 0, nv=(3, 4, 2), vl=2.0)
    rng = np.random.default_rng(2)
    f = rng.uniform(0.5, 1.5, (pr.npts, pr.nvel))
    R = pr.residual(f)
    F = f.reshape(tuple(ne[::-1]) + (pr.nvel,))  # [ez][ey][ex][k] (element-major, x fastest)
    h = [1.0 / n for n in ne]
    ref = np.zeros_like(F)
    for d in range(dim):
        ax = dim - 1 - d
        a = pr.xi[:, d]
        back = F - np.roll(F, 1, axis=ax)   # f_i - f_{i-1}
        fwd = np.roll(F, -1, axis=ax) - F   # f_{i+1} - f_i
        ref -= np.where(a > 0, a * back, a * fwd) / h[d]
    assert np.allclose(R, ref.reshape(R.shape), atol=1e-13, rtol=1e-13)


def _lagrange_polys(x):
    """Lagrange basis of the nodes x as numpy power-series coefficient arrays."""
    polys = []
    for j in range(len(x)):
        others = np.delete(x, j)
        c = nppoly.polyfromroots(others)
        polys.append(c / nppoly.polyval(x[j], c))
    return polys


@pytest.mark.parametrize("p", [1, 2, 3, 5])
def test_matches_weak_form_dg(p):
    # Independent formulation: nodal DG in weak form with exact mass and stiffness integrals,
    #   (h/2) M df/dt = a K f - l(1) F_R + l(-1) F_L,  M_ij = int l_i l_j, K_ij = int l_i' l_j,
    # with the upwind fluxes F_L, F_R. FR with g_DG must reproduce it (Sec. 2.1, Eq. 8).
    ne = 6
    pr = make(1, [ne], p, nv=(3, 2, 2), vl=1.5)
    x, _ = np.polynomial.legendre.leggauss(p + 1)
    L = _lagrange_polys(x)
    xq, wq = npleg.leggauss(2 * p + 4)
    V = np.array([nppoly.polyval(xq, c) for c in L])
    dV = np.array([nppoly.polyval(xq, nppoly.polyder(c)) for c in L])
    M = (V * wq) @ V.T
    K = (dV * wq) @ V.T
    lm = np.array([nppoly.polyval(-1.0, c) for c in L])
    lp = np.array([nppoly.polyval(1.0, c) for c in L])
    h = 1.0 / ne
    rng = np.random.default_rng(3)
    f = rng.uniform(0.2, 1.0, (pr.npts, pr.nvel))
    R = pr.residual(f)
    F = f.reshape(ne, p + 1, pr.nvel)
    ref = np.zeros_like(F)
    Minv = np.linalg.inv(M)
    for e in range(ne):
        for k in range(pr.nvel):
            a = pr.xi[k, 0]
            fe = F[e, :, k]
            left = F[(e - 1) % ne, :, k] @ lp     # neighbour trace at the shared left face
            right = F[(e + 1) % ne, :, k] @ lm
            FL = a * (left if a > 0 else fe @ lm)
            FR = a * (fe @ lp if a > 0 else right)
            ref[e, :, k] = (2.0 / h) * Minv @ (a * K @ fe - lp * FR + lm * FL)
    assert np.allclose(R, ref.reshape(R.shape), atol=1e-11, rtol=1e-11)


def _advect_error(dim, ne, p, T=0.1):
    pr = make(dim, [ne] * dim, p, nv=(2, 2, 2), vl=1.0)
    X = pr.points()
    s = X[:, :dim].sum(1)
    f0 = 1.0 + 0.5 * np.sin(2 * np.pi * s)
    pr.set_f(np.repeat(f0[:, None], pr.nvel, 1))
    h = 1.0 / ne
    nst = int(np.ceil(T / (0.02 * h)))
    pr.step(T / nst, nst)
    c = pr.xi[:, :dim].sum(1)
    exact = 1.0 + 0.5 * np.sin(2 * np.pi * (s[:, None] - c[None, :] * T))
    return np.abs(pr.get_f() - exact).max()


@pytest.mark.parametrize("p", [1, 2, 3])
def test_convergence_order_1d(p):
    # smooth periodic advection sin(2 pi (x - xi t)) converges at order p + 1
    e1, e2 = _advect_error(1, 8, p), _advect_error(1, 16, p)
    assert np.log2(e1 / e2) > p + 0.6


@pytest.mark.parametrize("p,ne", [(1, 8), (2, 6)])
def test_convergence_order_3d(p, ne):
    e1, e2 = _advect_error(3, ne, p, T=0.05), _advect_error(3, 2 * ne, p, T=0.05)
    assert np.log2(e1 / e2) > p + 0.6


def test_3d_equals_1d_for_x_only_data():
    # a state that varies only in x, periodic in y and z, evolves as the 1-D problem (including
    # collisions): checks the 3-D node/element indexing and the y/z fluxes cancelling.
    p, ne = 2, 4
    kw = dict(nv=(4, 4, 4), vl=3.0, tau=0.05)
    p1 = make(1, [ne], p, **kw)
    p3 = make(3, [ne, 2, 3], p, **kw)
    x1 = p1.points()[:, 0]
    prim1 = np.stack([1 + 0.2 * np.sin(2 * np.pi * x1), 0.1 * np.cos(2 * np.pi * x1),
                      0 * x1, 0 * x1, 1 + 0.1 * np.sin(2 * np.pi * x1)], 1)
    x3 = p3.points()[:, 0]
    prim3 = np.stack([1 + 0.2 * np.sin(2 * np.pi * x3), 0.1 * np.cos(2 * np.pi * x3),
                      0 * x3, 0 * x3, 1 + 0.1 * np.sin(2 * np.pi * x3)], 1)
    p1.set_state(prim1)
    p3.set_state(prim3)
    dt = 0.01
    p1.step(dt, 3)
    p3.step(dt, 3)
    f1 = p1.get_f()
    f3 = p3.get_f()
    # map every 3-D point to the 1-D point with the same x-node
    idx = np.array([np.argmin(np.abs(x1 - xx)) for xx in x3])
    assert np.allclose(f3, f1[idx], atol=1e-13, rtol=1e-12)


def test_2d_equals_1d_for_x_only_data():
    # quadrilaterals (dim = 2, 3-D velocity space): a state that varies only in x, periodic in y,
    # evolves as the line problem
    p, ne = 3, 4
    kw = dict(nv=(4, 4, 4), vl=3.0, tau=0.05)
    p1, p2 = make(1, [ne], p, **kw), make(2, [ne, 3], p, **kw)

    def prim(x):
        s = np.sin(2 * np.pi * x)
        return np.stack([1 + 0.2 * s, 0.1 * np.cos(2 * np.pi * x), 0.05 * s, 0 * x, 1 + 0.1 * s], 1)

    x1, x2 = p1.points()[:, 0], p2.points()[:, 0]
    p1.set_state(prim(x1))
    p2.set_state(prim(x2))
    p1.step(0.01, 3)
    p2.step(0.01, 3)
    idx = np.array([np.argmin(np.abs(x1 - xx)) for xx in x2])
    assert np.allclose(p2.get_f(), p1.get_f()[idx], atol=1e-13, rtol=1e-12)
