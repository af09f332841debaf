"""Oracle pins for curvilinear hexahedra (the metric terms of FR on mapped elements, Sec. 2.1, Eqs. 6-9
on a curved element: the reference-space flux (Ja^i . xi) f, the upwind flux with u_n = Ja^i . xi).

The metric terms are pinned against the closed-form cofactor matrix of a known quadratic mapping
(exact at p >= 2); the method against the affine path (the same mesh given as node coordinates), the
discrete metric identities and free-stream preservation, volume, conservation on a non-polynomial
(not watertight) mapping, the order of accuracy on a smooth curved geometry, and the J-weighted limiter
mean.
CPU only."""
import math

import numpy as np
import pytest

from oracle import oracle as orc
from paper_2308_06196_gb300 import workloads as W

L3 = (1.0, 1.0, 1.0)


def box(ne, p, n=4, L=3.0, tau=0.05, lo=(0.0,) * 3, hi=L3, **kw):
    return orc.Problem(3, list(ne), list(lo), list(hi), p, (n, n, n), (-L,) * 3, (L,) * 3, tau, **kw)


def bump_metric(x, lo, hi, ne, eps):
    """Closed form of the bump mapping's metric: d X / d r = A diag(h / 2) with A = I + E,
    E[d, d+1] = eps h_d 4 (1 - 2 t_{d+1}) / h_{d+1}; J = det, Ja[i, n] = J (dX/dr)^-1[i, n]."""
    lo, hi, ne = np.asarray(lo), np.asarray(hi), np.asarray(ne)
    h = (hi - lo) / ne
    Ja = np.zeros((len(x), 3, 3))
    J = np.zeros(len(x))
    for q, xq in enumerate(x):
        A = np.eye(3)
        for d in range(3):
            e = (d + 1) % 3
            t = (xq[e] - lo[e]) / h[e]
            tl = t - math.floor(t)
            A[d, e] = eps * h[d] * 4.0 * (1.0 - 2.0 * tl) / h[e]
        M = A @ np.diag(h / 2)
        J[q] = np.linalg.det(M)
        Ja[q] = J[q] * np.linalg.inv(M)
    return Ja, J


@pytest.mark.parametrize("p", [2, 3])
def test_metric_equals_closed_form_of_a_quadratic_mapping(p):
    ne, eps = (3, 2, 2), 0.15
    pr = box(ne, p)
    x = pr.points()
    pr.set_geometry(W.curved_nodes(x, (0, 0, 0), L3, ne, eps))
    Ja, J = pr.metric()
    Ja_ex, J_ex = bump_metric(x, (0, 0, 0), L3, ne, eps)
    # round-off of differentiating O(1) coordinates into O(h^3) and O(h^2) quantities
    assert np.abs(J - J_ex).max() <= 1e-13 * np.abs(J_ex).max()
    assert np.abs(Ja - Ja_ex).max() <= 1e-12 * np.abs(Ja_ex).max()
    assert J.std() > 1e-3 * J.mean()  # the mesh is genuinely curved


def test_affine_nodes_reproduce_the_affine_path():
    ne, p = (2, 3, 2), 2
    lo, hi = (0.0, -1.0, 0.5), (2.0, 1.0, 1.5)
    a, b = box(ne, p, lo=lo, hi=hi), box(ne, p, lo=lo, hi=hi)
    b.set_geometry(a.points())
    prim = W.smooth_prim(a.points(), 3, seed=2)
    a.set_state(prim)
    b.set_state(prim)
    f = a.get_f() * W.noise((a.npts, a.nvel), seed=3, amp=0.1)
    Ra, Rb = a.residual(f), b.residual(f)
    assert np.abs(Ra - Rb).max() <= 1e-12 * np.abs(Ra).max()
    assert a.dt(0.1) == pytest.approx(b.dt(0.1), rel=1e-13)
    a.set_f(f)
    b.set_f(f)
    a.step(0.01, 2)
    b.step(0.01, 2)
    assert np.abs(a.get_f() - b.get_f()).max() <= 1e-12 * np.abs(a.get_f()).max()


@pytest.mark.parametrize("p", [2, 3])
def test_metric_identities_and_free_stream(p):
    ne, eps = (2, 2, 2), 0.2
    pr = box(ne, p, tau=0.05)
    pr.set_geometry(W.curved_nodes(pr.points(), (0, 0, 0), L3, ne, eps))
    Ja, J = pr.metric()
    # sum_i d/dr_i (Ja^i_n) = 0 at every node (D applied along each reference direction)
    D = orc.fr_operators(p)[0]
    n1 = p + 1
    A = Ja.reshape(-1, n1, n1, n1, 3, 3)  # e, iz, iy, ix, i, n
    div = (np.einsum("ak,ezykn->ezyan", D, A[..., 0, :]) + np.einsum("ak,ezkxn->ezaxn", D, A[..., 1, :])
           + np.einsum("ak,ekyxn->eayxn", D, A[..., 2, :]))
    assert np.abs(div).max() <= 1e-13 * np.abs(Ja).max()
    # a spatially constant f: zero advection residual, and a uniform state stays uniform under RK3 + BGK
    g = pr.sample_maxwellian([1.0, 0.3, -0.2, 0.1, 0.9]) * W.noise(pr.nvel, seed=5, amp=0.2)
    F = np.tile(g, (pr.npts, 1))
    assert np.abs(pr.residual(F)).max() <= 1e-12 * g.max()
    pr.set_f(F)
    pr.step(pr.dt(0.1), 3)
    f = pr.get_f()
    assert np.abs(f - f[:1]).max() <= 1e-13 * g.max()


def test_bump_mapping_keeps_the_volume():
    ne = (3, 2, 2)
    pr = box(ne, 2)
    pr.set_geometry(W.curved_nodes(pr.points(), (0, 0, 0), L3, ne, 0.2))
    _, J = pr.metric()
    _, w = orc.gauss_legendre(3)
    Wn = np.einsum("i,j,k->kji", w, w, w).ravel()
    assert abs((J.reshape(-1, 27) * Wn).sum() - 1.0) <= 1e-14


def test_conservation_on_a_non_polynomial_mapping():
    # the sine mapping is not polynomial per element (neighbouring interpolants disagree at faces);
    # the single-valued face normal still makes the J-weighted totals conserved
    ne, p = (3, 2, 2), 2
    pr = box(ne, p, n=6, L=4.0, tau=0.02)
    pr.set_geometry(W.curved_nodes(pr.points(), (0, 0, 0), L3, ne, 0.3, kind="sine"))
    _, J = pr.metric()
    _, w = orc.gauss_legendre(p + 1)
    Wn = np.einsum("i,j,k->kji", w, w, w).ravel()
    WJ = (J.reshape(-1, Wn.size) * Wn).ravel()
    pr.set_state(W.smooth_prim(pr.points(), 3, seed=8, amp=0.2))
    T0 = (pr.moments() * WJ[:, None]).sum(0)
    pr.step(pr.dt(0.1), 10)
    T1 = (pr.moments() * WJ[:, None]).sum(0)
    assert np.abs(T1 - T0).max() <= 1e-12 * np.abs(T0).max()


def advection_error(p, ne, amp_geom=0.1, t_end=0.25):
    """J-weighted L2 error of pure advection (no collisions) of f0 = 1 + a_k sin(2 pi (x + y + z)), for
    the 8 velocities (+-1)^3 (a per-velocity amplitude a_k), against f0(x - xi t), on the sine mesh of a
    fixed geometry (displacement amplitude amp_geom for every ne). A fixed smooth geometry is what
    refinement resolves; elements that keep their curved shape as they shrink (curvature ~ 1/h, the bump
    family) converge at order p only, the known condition on curved element families."""
    pr = orc.Problem(3, [ne] * 3, [0.0] * 3, [1.0] * 3, p, (2, 2, 2), (-1.0,) * 3, (1.0,) * 3, math.inf)
    X = W.curved_nodes(pr.points(), (0, 0, 0), L3, (ne,) * 3, amp_geom * ne, kind="sine")
    pr.set_geometry(X)
    amp = 0.3 + 0.05 * np.arange(8)

    def exact(t):
        arg = ((X[:, None, :] - pr.xi[None, :, :] * t).sum(-1))
        return 1.0 + amp[None, :] * np.sin(2 * np.pi * arg)

    pr.set_f(exact(0.0))
    n = int(math.ceil(t_end / pr.dt(0.1)))
    pr.step(t_end / n, n)
    _, J = pr.metric()
    _, w = orc.gauss_legendre(p + 1)
    Wn = np.einsum("i,j,k->kji", w, w, w).ravel()
    WJ = (J.reshape(-1, Wn.size) * Wn).ravel()
    return math.sqrt((WJ[:, None] * (pr.get_f() - exact(t_end)) ** 2).sum())


@pytest.mark.parametrize("p", [2, 3])
def test_order_of_accuracy_on_a_curved_mesh(p):
    e1, e2 = advection_error(p, 3), advection_error(p, 6)
    assert math.log2(e1 / e2) > p + 0.5, (e1, e2)


def test_limiter_keeps_the_physical_element_mean():
    ne, p = (2, 2, 1), 2
    pr = box(ne, p, n=4)
    pr.set_geometry(W.curved_nodes(pr.points(), (0, 0, 0), L3, ne, 0.25))
    _, J = pr.metric()
    _, w = orc.gauss_legendre(p + 1)
    Wn = np.einsum("i,j,k->kji", w, w, w).ravel()
    f = np.random.default_rng(9).uniform(-0.5, 2.0, size=(pr.npts, pr.nvel))
    g = pr.limit(f)
    WJ = (J.reshape(-1, Wn.size) * Wn)
    mean = lambda a: np.einsum("ei,eik->ek", WJ, a.reshape(-1, Wn.size, pr.nvel)) / WJ.sum(1)[:, None]
    assert np.abs(mean(g) - mean(f)).max() <= 1e-14 * np.abs(mean(f)).max()
    neg = f.reshape(-1, Wn.size, pr.nvel).min(1) < 0
    ok = neg & (mean(f) >= 0)
    assert np.abs(g.reshape(-1, Wn.size, pr.nvel).min(1)[ok]).max() <= 1e-14


# ------------------------------------------------------------------------------------------------
# unstructured connectivity: the structured grid relabelled (random element order, every element's
# local axes rotated at random) is the same discretisation, so it must reproduce the structured
# result point for point; a wrong orientation bit, trace end or normal sign anywhere breaks this


@pytest.mark.parametrize("kind,bc", [("bump", None), ("sine", "tube")])
def test_unstructured_relabelling_reproduces_the_structured_mesh(kind, bc):
    ne, p = (3, 2, 2), 2
    bcs = None
    if bc == "tube":
        bc = np.array([[W.DIRICHLET, W.DIRICHLET], [0, 0], [0, 0]])
        bcs = np.zeros((3, 2, 5))
        bcs[0, 0] = [1.0, 0.3, 0.0, 0.0, 1.0]
        bcs[0, 1] = [0.5, 0.3, 0.0, 0.0, 0.9]
    u = W.unstructured_box(ne, p, bc=None if bc is None else bc.tolist(), seed=5)
    kw = dict(bc=None if bc is None else bc.reshape(6), bc_state=None if bcs is None else bcs.reshape(30))
    a, b = box(ne, p, n=6, L=4.0, tau=0.05, **kw), box(ne, p, n=6, L=4.0, tau=0.05, **kw)
    X = W.curved_nodes(a.points(), (0, 0, 0), L3, ne, 0.3 if kind == "sine" else 0.15, kind=kind)
    m = u["node_map"]
    a.set_geometry(X)
    b.set_connectivity(u["nbr"], u["nface"], u["orient"])
    b.set_geometry(X[m])
    assert b.dt(0.1) == pytest.approx(a.dt(0.1), rel=1e-13)
    prim = W.smooth_prim(X, 3, seed=2)
    a.set_state(prim)
    f = a.get_f() * W.noise((a.npts, a.nvel), seed=3, amp=0.1)
    Ra, Rb = a.residual(f), b.residual(f[m])
    assert np.abs(Ra[m] - Rb).max() <= 1e-13 * np.abs(Ra).max()
    a.set_f(f)
    b.set_f(f[m])
    a.set_limiter(True)
    b.set_limiter(True)
    a.step(0.01, 3)
    b.step(0.01, 3)
    assert np.abs(a.get_f()[m] - b.get_f()).max() <= 1e-13 * np.abs(a.get_f()).max()


def test_unstructured_tables_are_validated():
    pr = box((2, 2, 2), 2)
    u = W.unstructured_box((2, 2, 2), 2, seed=1)
    bad = u["orient"].copy()
    bad[0, 0] = 9
    with pytest.raises(ValueError):
        pr.set_connectivity(u["nbr"], u["nface"], bad)
    nb = u["nbr"].copy()
    nb[0, 0] = -1  # a boundary face on a periodic grid: no Dirichlet or wall data for it
    with pytest.raises(ValueError):
        pr.set_connectivity(nb, u["nface"], u["orient"])


# ------------------------------------------------------------------------------------------------
# diffuse walls on curved faces: the wall density of every face point makes the net discrete mass
# flux through the curved face's own normal vanish


def channel(ne, p, n=6, L=4.0, tau=0.05):
    bc = np.array([[0, 0], [orc.WALL, orc.WALL], [0, 0]]).reshape(6)
    bcs = np.zeros((3, 2, 5))
    bcs[1, 0] = [0, 0.0, 0.0, 0.0, 1.0]
    bcs[1, 1] = [0, 0.2, 0.0, 0.0, 1.0]  # the upper wall moves in x
    return box(ne, p, n=n, L=L, tau=tau, bc=bc, bc_state=bcs.reshape(30))


def test_affine_nodes_with_walls_reproduce_the_affine_path():
    ne, p = (2, 3, 2), 2
    a, b = channel(ne, p), channel(ne, p)
    b.set_geometry(a.points())
    a.set_state(W.smooth_prim(a.points(), 3, seed=3))
    f = a.get_f() * W.noise((a.npts, a.nvel), seed=4, amp=0.1)
    Ra, Rb = a.residual(f), b.residual(f)
    assert np.abs(Ra - Rb).max() <= 1e-12 * np.abs(Ra).max()


def test_curved_walls_conserve_mass():
    # walls at y = 0 and y = 1 made wavy by the sine mapping (x and z periodic): the J-weighted total
    # mass is conserved to round-off; momentum and energy exchange with the walls
    ne, p = (3, 3, 2), 2
    pr = channel(ne, p, tau=0.02)
    X = W.curved_nodes(pr.points(), (0, 0, 0), L3, ne, 0.3, kind="sine")
    pr.set_geometry(X)
    _, J = pr.metric()
    _, w = orc.gauss_legendre(p + 1)
    Wn = np.einsum("i,j,k->kji", w, w, w).ravel()
    WJ = (J.reshape(-1, Wn.size) * Wn).ravel()
    pr.set_state(W.smooth_prim(X, 3, seed=5, amp=0.2))
    T0 = (pr.moments() * WJ[:, None]).sum(0)
    pr.step(pr.dt(0.1), 10)
    T1 = (pr.moments() * WJ[:, None]).sum(0)
    assert abs(T1[0] - T0[0]) <= 1e-12 * T0[0]
    assert abs(T1[1] - T0[1]) > 1e-6 * T0[0]  # the moving wall drags the gas


def test_unstructured_walls_reproduce_the_structured_channel():
    # the wavy-walled channel (moving upper wall) relabelled and rotated: the walls are boundary faces of
    # the tables, in whatever local face they fall; point for point equal to the structured run
    ne, p = (3, 3, 2), 2
    bcw = [[0, 0], [orc.WALL, orc.WALL], [0, 0]]
    u = W.unstructured_box(ne, p, bc=bcw, seed=9)
    m = u["node_map"]
    a, b = channel(ne, p, tau=0.02), channel(ne, p, tau=0.02)
    X = W.curved_nodes(a.points(), (0, 0, 0), L3, ne, 0.3, kind="sine")
    a.set_geometry(X)
    b.set_connectivity(u["nbr"], u["nface"], u["orient"])
    b.set_geometry(X[m])
    a.set_state(W.smooth_prim(X, 3, seed=6, amp=0.2))
    f = a.get_f()
    b.set_f(f[m])
    Ra, Rb = a.residual(f), b.residual(f[m])
    assert np.abs(Ra[m] - Rb).max() <= 1e-13 * np.abs(Ra).max()
    a.step(0.01, 3)
    b.step(0.01, 3)
    assert np.abs(a.get_f()[m] - b.get_f()).max() <= 1e-13 * np.abs(a.get_f()).max()
