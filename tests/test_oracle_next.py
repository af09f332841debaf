"""Oracle pins for the widened rows of the method: the Zhang-Shu positivity limiter (Sec. 2.1,
Eqs. 10-11) and the non-conservative ablation, where the BGK source relaxes towards the sampled
continuous Maxwellian of the moments instead of the discretely-conservative one (Sec. 2.1, Eq. 13 and
the text after it)."""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_2308_06196_gb300 import workloads as W


def gl_weights_tensor(p, dim):
    _, w = orc.gauss_legendre(p + 1)
    if dim == 1:
        return w
    return np.einsum("i,j,k->kji", w, w, w).ravel()


# ------------------------------------------------------------------------------------------------
# positivity limiter


def test_limiter_worked_example():
    # one p = 1 line element (two Gauss-Legendre nodes of equal weight), f = (-1, 3) at one velocity:
    # mean 1, min -1, beta = |1 / (1 - (-1))| = 1/2, so f -> 1 + (f - 1) / 2 = (0, 2); a velocity with
    # f = (2, 5) has no negative value and is left alone
    pr = orc.Problem(1, [1], [0.0], [1.0], 1, (4, 4, 4), (-3.0,) * 3, (3.0,) * 3, 0.1)
    f = np.ones((pr.npts, pr.nvel))
    f[:, 0] = [-1.0, 3.0]
    f[:, 1] = [2.0, 5.0]
    g = pr.limit(f)
    assert np.array_equal(g[:, 0], [0.0, 2.0])
    assert np.array_equal(g[:, 1:], f[:, 1:])


@pytest.mark.parametrize("dim,p", [(1, 3), (3, 2)])
def test_limiter_keeps_means_and_restores_positivity(dim, p):
    ne = [5] if dim == 1 else [2, 2, 1]
    pr = orc.Problem(dim, ne, [0.0] * dim, [1.0] * dim, p, (6, 6, 6), (-4.0,) * 3, (4.0,) * 3, 0.1)
    rng = np.random.default_rng(4)
    f = rng.uniform(-0.5, 2.0, size=(pr.npts, pr.nvel))
    g = pr.limit(f)
    Wn = gl_weights_tensor(p, dim)
    np_ = len(Wn)
    fe, ge = f.reshape(-1, np_, pr.nvel), g.reshape(-1, np_, pr.nvel)
    mean_f = np.einsum("i,eik->ek", Wn, fe) / Wn.sum()
    mean_g = np.einsum("i,eik->ek", Wn, ge) / Wn.sum()
    assert np.abs(mean_g - mean_f).max() <= 1e-14 * np.abs(mean_f).max()
    neg = fe.min(axis=1) < 0
    # where the mean is non-negative, the limited values are (up to round-off) non-negative and the
    # smallest one is 0
    ok = neg & (mean_f >= 0)
    assert ge.min(axis=1)[ok].min() >= -1e-14
    assert np.abs(ge.min(axis=1)[ok]).max() <= 1e-14
    # (element, velocity) pairs without a negative value are untouched
    assert np.array_equal(ge.transpose(0, 2, 1)[~neg], fe.transpose(0, 2, 1)[~neg])


def sod(p=3, E=12, N=12, tau=1e-3, jump=(1.0, 1.0, 0.125, 0.8)):
    rl, tl, rr, tr = jump
    bc = np.array([[W.DIRICHLET, W.DIRICHLET], [0, 0], [0, 0]]).reshape(6)
    bcs = np.zeros((3, 2, 5))
    bcs[0, 0] = [rl, 0, 0, 0, tl]
    bcs[0, 1] = [rr, 0, 0, 0, tr]
    pr = orc.Problem(1, [E], [0.0], [1.0], p, (N, N, N), (-8.0,) * 3, (8.0,) * 3, tau, bc=bc, bc_state=bcs.reshape(30))
    pr.set_state(W.prim_sod(pr.points(), (rl, tl), (rr, tr)))
    return pr


def positivity(pr, f):
    """(smallest f / element mean over the (element, velocity) pairs with a non-negative mean,
    most negative element mean, relative to max f)."""
    Wn = gl_weights_tensor(pr.p, pr.dim)
    fe = f.reshape(-1, len(Wn), pr.nvel)
    mean = np.einsum("i,eik->ek", Wn, fe) / Wn.sum()
    pos = mean > 0
    return (fe.min(axis=1)[pos] / mean[pos]).min(), min(mean.min(), 0.0) / f.max()


def test_limiter_keeps_a_shock_tube_positive():
    # a strong density jump at p = 3 under-shoots without the limiter; with it, every node value is
    # >= 0 wherever the element mean is (the limiter keeps means, so a mean that advection made
    # negative, here only in the far velocity tails at round-off size, stays negative)
    plain, limited = sod(), sod()
    limited.set_limiter(True)
    dt = plain.dt(0.1)
    min_plain = 0.0
    for _ in range(10):
        plain.step(dt, 1)
        limited.step(dt, 1)
        f = plain.get_f()
        min_plain = min(min_plain, f.min() / f.max())
        ratio, neg_mean = positivity(limited, limited.get_f())
        assert ratio >= -1e-12
        assert neg_mean >= -1e-10
    assert min_plain < -1e-5


def test_limiter_conserves_on_a_periodic_line():
    # the limiter keeps every element mean, so the periodic totals stay constant to round-off
    p, ne = 3, 8
    pr = orc.Problem(1, [ne], [0.0], [1.0], p, (10, 10, 10), (-5.0,) * 3, (5.0,) * 3, 0.01)
    x = pr.points()[:, 0]
    P = np.zeros((pr.npts, 5))
    P[:, 0] = np.where((x > 0.3) & (x < 0.6), 1.0, 0.05)
    P[:, 4] = 1.0
    pr.set_state(P)
    pr.set_limiter(True)
    Wn = gl_weights_tensor(p, 1)

    def tot(Q):
        return (Q.reshape(ne, p + 1, 5) * Wn[None, :, None]).sum((0, 1))

    T0 = tot(pr.moments())
    pr.step(pr.dt(0.1), 40)
    ratio, neg_mean = positivity(pr, pr.get_f())
    assert ratio >= -1e-12 and neg_mean >= -1e-9
    assert np.abs(tot(pr.moments()) - T0).max() <= 1e-12 * np.abs(T0).max()


# ------------------------------------------------------------------------------------------------
# non-conservative ablation (continuous Maxwellian)


def state_of(Q):
    rho = Q[:, 0]
    U = Q[:, 1:4] / rho[:, None]
    th = (2.0 / 3.0) * (Q[:, 4] / rho - 0.5 * (U**2).sum(1))
    return np.column_stack([rho, U, th])


def test_continuous_equilibrium_is_the_state_of_the_moments():
    pr = orc.Problem(1, [3], [0.0], [1.0], 2, (8, 8, 8), (-5.0,) * 3, (5.0,) * 3, 0.1)
    pr.set_state(W.smooth_prim(pr.points(), 1, seed=2, amp=0.3))
    Q = pr.moments()
    pr.set_maxwellian(True)
    P, it, res, bad = pr.conservative_maxwellian(Q)
    assert bad == 0
    assert np.abs(P - state_of(Q)).max() <= 1e-14 * np.abs(state_of(Q)).max()


def drift(N, continuous, steps=20):
    # space-homogeneous relaxation of a two-stream state: every change of the moments is the BGK
    # source's conservation error (velocity domain wide enough that truncation plays no part)
    pr = orc.Problem(1, [1], [0.0], [1.0], 1, (N, N, N), (-10.0,) * 3, (10.0,) * 3, 1e-2)
    a = pr.sample_maxwellian([1.0, 0.8, 0.0, 0.0, 0.6])
    b = pr.sample_maxwellian([0.5, -1.2, 0.3, 0.0, 0.9])
    pr.set_f(np.tile(a + b, (pr.npts, 1)))
    pr.set_maxwellian(continuous)
    Q0 = pr.moments()
    pr.step(5e-3, steps)
    return np.abs(pr.moments() - Q0).max() / np.abs(Q0).max()


def test_continuous_maxwellian_breaks_conservation_and_the_error_falls_with_resolution():
    cons = drift(10, False)
    d10, d16, d24 = drift(10, True), drift(16, True), drift(24, True)
    assert cons <= 1e-12
    # the ablation's conservation error is far above round-off on a coarse grid and falls quickly as
    # the trapezoid rule resolves the Maxwellians (spectral convergence)
    assert d10 > 1e-2
    assert d16 < d10 / 10 and d24 < d16 / 1e3


def test_conservative_state_tends_to_the_moments_state():
    # the perturbed state Q' of the conservative Maxwellian converges to the state of Q as the
    # velocity grid is refined
    gaps = []
    for N in (8, 12, 16, 24):
        pr = orc.Problem(1, [1], [0.0], [1.0], 1, (N, N, N), (-6.0,) * 3, (6.0,) * 3, 0.1)
        a = pr.sample_maxwellian([1.0, 0.3, 0.0, 0.0, 0.8])
        Q = pr.moments(np.tile(a, (pr.npts, 1)))
        P, _, _, bad = pr.conservative_maxwellian(Q)
        assert bad == 0
        gaps.append(np.abs(P - state_of(Q)).max())
    assert gaps[1] < gaps[0] and gaps[2] < gaps[1] and gaps[3] < gaps[2]
    assert gaps[3] < 1e-6 * gaps[0]


# ------------------------------------------------------------------------------------------------
# variable collision time tau = mu(theta) / P (Sec. 2, Eq. 5)


@pytest.mark.parametrize("rho,th", [(1.0, 1.0), (0.3, 1.6)])
def test_variable_tau_space_homogeneous_closed_form(rho, th):
    # a uniform non-equilibrium state keeps its moments, hence its tau = mu_ref theta^omega / P;
    # the Shu-Osher steps of the linear relaxation then give f_n = M + (f_0 - M) R(-dt/tau)^n with
    # R(z) = 1 + z + z^2/2 + z^3/6 exactly
    mu_ref, omega = 2e-3, 0.81
    pr = orc.Problem(1, [1], [0.0], [1.0], 1, (12, 12, 12), (-7.0,) * 3, (7.0,) * 3, 1.0)
    a = pr.sample_maxwellian([rho, 0.3, 0.0, 0.0, th])
    b = pr.sample_maxwellian([0.2 * rho, -1.0, 0.5, 0.0, 0.5 * th])
    f0 = a + b
    Q = pr.moments(np.tile(f0, (pr.npts, 1)))[0]
    state = state_of(Q[None])[0]  # the mixture's (rho, U, theta): P = rho theta of it
    tau = mu_ref * state[4] ** omega / (state[0] * state[4])
    pr.set_newton(1e-14, 50)
    P, _, _, bad = pr.conservative_maxwellian(Q[None])
    assert bad == 0
    M = pr.sample_maxwellian(P[0])
    pr.set_f(np.tile(f0, (pr.npts, 1)))
    pr.set_viscosity(mu_ref, omega)
    dt, n = 0.4 * tau, 7
    pr.step(dt, n)
    z = -dt / tau
    R = 1 + z + z * z / 2 + z**3 / 6
    exact = M + (f0 - M) * R**n
    assert np.abs(pr.get_f()[0] - exact).max() <= 1e-12 * f0.max()


def test_variable_tau_differs_between_states_and_conserves():
    # a periodic line with a density step: tau varies along the line (1 / rho), the totals stay
    # constant to round-off
    p, ne = 2, 6
    pr = orc.Problem(1, [ne], [0.0], [1.0], p, (10, 10, 10), (-6.0,) * 3, (6.0,) * 3, 1.0)
    x = pr.points()[:, 0]
    P = np.zeros((pr.npts, 5))
    P[:, 0] = np.where(x < 0.5, 1.0, 0.25)
    P[:, 1] = 0.2
    P[:, 4] = np.where(x < 0.5, 1.0, 1.5)
    pr.set_state(P)
    pr.set_viscosity(5e-3, 0.75)
    _, w = orc.gauss_legendre(p + 1)

    def tot(Q):
        return (Q.reshape(ne, p + 1, 5) * w[None, :, None]).sum((0, 1))

    T0 = tot(pr.moments())
    pr.step(2e-3, 30)
    assert np.abs(tot(pr.moments()) - T0).max() <= 1e-12 * np.abs(T0).max()
