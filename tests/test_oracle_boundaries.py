"""Pins of the oracle's boundary faces against closed forms and brute force (CPU only).

The upwind common flux (paper Sec. 2.1, Eq. 9) takes the exterior value only where the face flow
enters the element; at a Dirichlet face that exterior value is the sampled Maxwellian of the face's
prescribed state, and at a diffuse wall it is the wall Maxwellian (Eq. 4 with the wall's velocity
U_w and temperature T_w) scaled by the wall density of zero net discrete mass flux. These tests fix
which end's ghost is used, that it is used on inflow faces only, and the wall-velocity term."""
import numpy as np
import pytest
from numpy.polynomial import legendre as npleg

from oracle import oracle as orc

INF = float("inf")


def maxwell(xi, rho, U, th):
    # Eq. 4 with the velocity dimension 3, written out here for the expected values
    return rho / (2 * np.pi * th) ** 1.5 * np.exp(-((xi - np.asarray(U)) ** 2).sum(1) / (2 * th))


def radau_derivatives(p, x):
    """g_L'(x), g_R'(x) of the left/right Radau correction polynomials of degree p + 1 (Huynh's g_DG):
    g_L = (-1)^(p+1)/2 (P_{p+1} - P_p), g_R = (P_{p+1} + P_p)/2, differentiated as Legendre series."""
    cp1 = np.zeros(p + 2)
    cp1[p + 1] = 1.0
    cp = np.zeros(p + 2)
    cp[p] = 1.0
    gl = 0.5 * (-1) ** (p + 1) * (cp1 - cp)
    gr = 0.5 * (cp1 + cp)
    return npleg.legval(x, npleg.legder(gl)), npleg.legval(x, npleg.legder(gr))


# two different prescribed states at the two x ends (rho, u, v, w, T)
LO = [1.3, 0.4, -0.2, 0.1, 0.9]
HI = [0.6, -0.3, 0.15, -0.05, 1.4]


def dirichlet_x(dim, ne, p, nv=(6, 5, 4), L=4.0, tau=INF):
    bc = np.zeros(6, np.int32)
    bc[0] = bc[1] = orc.DIRICHLET
    bcs = np.zeros((6, 5))
    bcs[0], bcs[1] = LO, HI
    lo, hi = [0.0] * dim, [1.0] * dim
    return orc.Problem(dim, list(ne), lo, hi, p, nv, (-L, -L + 0.5, -L), (L, L, L - 0.5), tau, bc=bc, bc_state=bcs)


@pytest.mark.parametrize("dim", [1, 3])
def test_p0_dirichlet_is_upwind_fv_with_the_inflow_ghost(dim):
    # p = 0: FR is the textbook first-order upwind finite-volume difference per direction. At the x ends
    # the upwind value of the boundary cell is the ghost of THAT end (the low end's state at x = 0, the
    # high end's at x = 1) and only where xi_x points into the domain; the outflow face takes the cell's
    # own value. y and z are periodic.
    ne = [6] if dim == 1 else [5, 3, 4]
    pr = dirichlet_x(dim, ne, 0)
    rng = np.random.default_rng(21)
    f = rng.uniform(0.05, 0.5, (pr.npts, pr.nvel))
    R = pr.residual(f)
    F = f.reshape(tuple(ne[::-1]) + (pr.nvel,))
    gl, gh = maxwell(pr.xi, LO[0], LO[1:4], LO[4]), maxwell(pr.xi, HI[0], HI[1:4], HI[4])
    h = [1.0 / n for n in ne]
    ref = np.zeros_like(F)
    for d in range(dim):
        ax = dim - 1 - d
        a = pr.xi[:, d]
        left = np.roll(F, 1, axis=ax)     # upwind value for a > 0
        right = np.roll(F, -1, axis=ax)   # upwind value for a < 0
        if d == 0:
            idx0 = [slice(None)] * (dim + 1)
            idx0[ax] = 0
            left[tuple(idx0)] = gl         # the low end's ghost enters the first cell
            idxn = [slice(None)] * (dim + 1)
            idxn[ax] = ne[0] - 1
            right[tuple(idxn)] = gh        # the high end's ghost enters the last cell
        ref -= np.where(a > 0, a * (F - left), a * (right - F)) / h[d]
    assert np.allclose(R, ref.reshape(R.shape), atol=1e-13, rtol=1e-12)


@pytest.mark.parametrize("dim,p", [(1, 1), (1, 2), (1, 3), (3, 2)])
def test_dirichlet_closed_form_on_a_constant_interior(dim, p):
    # tau = inf and f = c_k constant in space: interior faces carry no jump, so only the boundary
    # elements' inflow faces act. With the ghost b of the face, the residual there is the correction
    #   R_i = -(2/h) xi_x (b - c) g_L'(x_i)  (low end, xi_x > 0),  -(2/h) xi_x (b - c) g_R'(x_i)  (high end,
    # xi_x < 0), and exactly zero wherever the boundary face is an outflow face.
    ne = [5] if dim == 1 else [4, 2, 3]
    pr = dirichlet_x(dim, ne, p)
    n1 = p + 1
    rng = np.random.default_rng(22)
    c = rng.uniform(0.05, 0.3, pr.nvel)
    f = np.tile(c, (pr.npts, 1))
    R = pr.residual(f)
    x, _ = npleg.leggauss(n1)
    dgl, dgr = radau_derivatives(p, x)
    b_lo = maxwell(pr.xi, LO[0], LO[1:4], LO[4])
    b_hi = maxwell(pr.xi, HI[0], HI[1:4], HI[4])
    a = pr.xi[:, 0]
    h = 1.0 / ne[0]
    # expected residual per x-element column and x-node (it does not depend on y, z nodes)
    exp = np.zeros((ne[0], n1, pr.nvel))
    exp[0] = -(2.0 / h) * np.where(a > 0, a * (b_lo - c), 0.0)[None, :] * dgl[:, None]
    exp[-1] = exp[-1] - (2.0 / h) * np.where(a < 0, a * (b_hi - c), 0.0)[None, :] * dgr[:, None]
    if dim == 1:
        Rr = R.reshape(ne[0], n1, pr.nvel)
        assert np.allclose(Rr, exp, atol=1e-12, rtol=1e-11)
    else:
        # node order: element-major (x fastest), node index x fastest
        Rr = R.reshape(ne[2], ne[1], ne[0], n1, n1, n1, pr.nvel)
        for ez in range(ne[2]):
            for ey in range(ne[1]):
                for iz in range(n1):
                    for iy in range(n1):
                        assert np.allclose(Rr[ez, ey, :, iz, iy, :, :], exp, atol=1e-12, rtol=1e-11)


def test_dirichlet_swapped_ends_would_be_detected():
    # the closed form above distinguishes the two ends: the low and high ghosts differ at every
    # velocity by far more than the tolerance, so a residual built from the swapped ghosts fails it
    pr = dirichlet_x(1, [5], 2)
    b_lo = maxwell(pr.xi, LO[0], LO[1:4], LO[4])
    b_hi = maxwell(pr.xi, HI[0], HI[1:4], HI[4])
    assert np.abs(b_lo - b_hi).max() > 1e3 * 1e-12 * np.abs(b_lo).max()
    # and the oracle's residual of a constant state matches the unswapped form only
    c = np.full(pr.nvel, 0.1)
    R = pr.residual(np.tile(c, (pr.npts, 1))).reshape(5, 3, pr.nvel)
    x, _ = npleg.leggauss(3)
    dgl, _ = radau_derivatives(2, x)
    a = pr.xi[:, 0]
    swapped = -(2.0 / 0.2) * np.where(a > 0, a * (b_hi - c), 0.0)[None, :] * dgl[:, None]
    assert not np.allclose(R[0], swapped, atol=1e-12, rtol=1e-11)


def channel(nv, uw_lo, uw_hi, tw_lo=1.1, tw_hi=1.1, ne=(2, 3, 2), p=2, L=(5.0, 6.0, 5.0), tau=INF):
    """Walls at y = 0 and y = 1 (periodic x, z), wall velocities uw_* (tangential) and temperatures."""
    bc = np.zeros(6, np.int32)
    bc[2] = bc[3] = orc.WALL
    bcs = np.zeros((6, 5))
    bcs[2] = [0.0, uw_lo[0], 0.0, uw_lo[2], tw_lo]
    bcs[3] = [0.0, uw_hi[0], 0.0, uw_hi[2], tw_hi]
    # x and z extents asymmetric (the wall velocity must not hide behind a symmetric grid); y symmetric
    vlo = (-L[0] + 0.7, -L[1], -L[2] + 0.4)
    vhi = (L[0] + 0.3, L[1], L[2] - 0.2)
    return orc.Problem(3, list(ne), [0.0] * 3, [1.0] * 3, p, nv, vlo, vhi, tau, bc=bc, bc_state=bcs)


def test_moving_walls_keep_the_gas_of_their_own_velocity_exactly():
    # a uniform Maxwellian at (rho, U_w, T_w) between walls that move tangentially at U_w with
    # temperature T_w is a fixed point of the diffuse wall: on a velocity grid symmetric in the wall
    # normal the zero-mass-flux density is rho, the ghost equals the interior trace, and the residual
    # vanishes to round-off. A dropped or sign-flipped U_w (or a swapped tangential component) gives a
    # ghost far from the interior.
    Uw = (0.35, 0.0, -0.25)
    pr = channel((10, 12, 9), Uw, Uw)
    st = [1.3, Uw[0], 0.0, Uw[2], 1.1]
    pr.set_state(np.tile(st, (pr.npts, 1)))
    f = pr.get_f()
    R = pr.residual(f)
    scale = np.abs(f).max() * 6.0 * 2 * 3 * 9
    assert np.abs(R).max() <= 1e-13 * scale
    for wrong in ([0.0, 0.0, 0.0], [-Uw[0], 0.0, -Uw[2]], [Uw[2], 0.0, Uw[0]]):
        g = maxwell(pr.xi, 1.3, wrong, 1.1)
        assert np.abs(g - f[0]).max() > 1e5 * 1e-13 * np.abs(f).max()


def test_moving_wall_drags_the_gas_by_the_half_range_flux():
    # gas at rest at the walls' temperature; the upper wall moves in x at U_w, the lower one is at rest.
    # The first-step rate of change of the total x-momentum is what the walls' incoming half-range
    # Maxwellians carry in beyond the gas's own flux: per wall, the sum over its inflow velocities of
    # w |xi_y| xi_x (rho_w M(U_w, T_w) - f), times the wall area (interior faces cancel). Its leading
    # order is rho U_w sqrt(T_w / 2 pi): the sign and size of the drag.
    Uw, T, rho = 0.3, 1.0, 1.0
    nv = (14, 40, 6)
    pr = channel(nv, (0.0, 0.0, 0.0), (Uw, 0.0, 0.0), tw_lo=T, tw_hi=T, L=(6.0, 6.0, 5.0))
    pr.set_state(np.tile([rho, 0.0, 0.0, 0.0, T], (pr.npts, 1)))
    f = pr.get_f()
    R = pr.residual(f)
    ne, n1 = (2, 3, 2), 3
    _, wg = npleg.leggauss(n1)
    Wn = np.einsum("i,j,k->kji", wg, wg, wg).ravel()
    vol = 1.0 / (ne[0] * ne[1] * ne[2]) / 8.0  # element volume over the reference cube's 8
    rate = (((R @ (pr.w * pr.xi[:, 0])).reshape(-1, Wn.size)) * Wn).sum() * vol
    # brute force of the two walls (area 1 x 1 each): wall densities of zero net discrete mass flux,
    # then the incoming half-range momentum flux of ghost minus gas
    fin, xy = f[0], pr.xi[:, 1]
    expect = 0.0
    for Uwall, inflow, outflow in (((0.0, 0.0, 0.0), xy > 0, xy < 0), ((Uw, 0.0, 0.0), xy < 0, xy > 0)):
        Mw = maxwell(pr.xi, 1.0, Uwall, T)
        rho_w = (pr.w * np.abs(xy) * fin)[outflow].sum() / (pr.w * np.abs(xy) * Mw)[inflow].sum()
        expect += (pr.w * np.abs(xy) * pr.xi[:, 0] * (rho_w * Mw - fin))[inflow].sum()
    assert rate > 0
    assert abs(rate - expect) <= 1e-10 * abs(expect)
    cont = rho * Uw * np.sqrt(T / (2 * np.pi))
    assert abs(rate - cont) <= 0.03 * cont
