"""Pins of the oracle's reference-element operators and velocity grid against closed forms and
library routines (paper Sec. 2.1, Eqs. 7-8 and Eq. 12). CPU only."""
import numpy as np
import pytest

from oracle import oracle as orc


@pytest.mark.parametrize("n", range(1, 10))
def test_gauss_legendre_matches_numpy(n):
    # the oracle finds the roots of P_n by Newton; numpy solves the Golub-Welsch eigenproblem
    x, w = orc.gauss_legendre(n)
    X, W = np.polynomial.legendre.leggauss(n)
    assert np.allclose(x, X, atol=1e-14, rtol=0)
    assert np.allclose(w, W, atol=1e-14, rtol=0)


@pytest.mark.parametrize("p", range(0, 7))
def test_derivative_matrix_exact_on_polynomials(p):
    D, lm, lp, dgl, dgr = orc.fr_operators(p)
    x, _ = orc.gauss_legendre(p + 1)
    for m in range(p + 1):
        dexact = m * x ** (m - 1) if m > 0 else np.zeros_like(x)
        assert np.allclose(D @ x**m, dexact, atol=1e-12)
        # end interpolants reproduce x^m at -1 and +1
        assert abs(lm @ x**m - (-1.0) ** m) < 1e-13
        assert abs(lp @ x**m - 1.0) < 1e-13


@pytest.mark.parametrize("p", range(0, 7))
def test_summation_by_parts(p):
    # sum_i W_i D_ij = l_j(1) - l_j(-1): integrating a derivative exactly (degree p - 1 <= 2p + 1)
    D, lm, lp, _, _ = orc.fr_operators(p)
    _, W = orc.gauss_legendre(p + 1)
    assert np.allclose(W @ D, lp - lm, atol=1e-12)


@pytest.mark.parametrize("p", range(0, 7))
def test_correction_equals_dg_lift(p):
    # FR with the Radau (g_DG) correction functions is nodal DG: with the exact, diagonal GL mass
    # matrix the DG surface lift at node i is l_i(-1) / W_i (left face) and l_i(+1) / W_i (right).
    # The oracle builds g' from Legendre derivatives, so this ties the two formulations together.
    _, lm, lp, dgl, dgr = orc.fr_operators(p)
    _, W = orc.gauss_legendre(p + 1)
    assert np.allclose(dgl, -lm / W, atol=1e-12)
    assert np.allclose(dgr, lp / W, atol=1e-12)
    assert abs(W @ dgl + 1.0) < 1e-13 and abs(W @ dgr - 1.0) < 1e-13


def test_velocity_grid_trapezoid():
    nv = (5, 6, 7)
    xi, w = orc.velocity_grid(nv, (-1.0, -2.0, -3.0), (1.0, 2.0, 3.0))
    assert xi.shape == (5 * 6 * 7, 3)
    # endpoints included, k = kx + nx*(ky + ny*kz)
    assert np.allclose(xi[0], (-1, -2, -3)) and np.allclose(xi[-1], (1, 2, 3))
    assert np.allclose(xi[1, 0] - xi[0, 0], 0.5) and np.allclose(xi[5, 1] - xi[0, 1], 0.8)
    assert abs(w.sum() - 2 * 4 * 6) < 1e-12
    # exact for linear functions (trapezoid rule), and a half weight at a corner
    assert abs((w * xi[:, 0]).sum()) < 1e-13
    assert abs(w[0] - 0.5 * 0.8 * 1.0 / 8) < 1e-15  # (dx/2)(dy/2)(dz/2)


def test_velocity_grid_spectral_gaussian():
    # trapezoid rule on a smooth, effectively compactly supported integrand is spectrally accurate
    # (Sec. 2.1, Eq. 12): the error of int exp(-|xi|^2/2) is the tail beyond the box, ~exp(-L^2/2)
    for n, L in ((16, 6.0), (24, 6.0), (24, 8.0)):
        xi, w = orc.velocity_grid((n, n, n), (-L,) * 3, (L,) * 3)
        val = (w * np.exp(-0.5 * (xi**2).sum(1))).sum()
        exact = (2 * np.pi) ** 1.5
        tail = 3 * np.sqrt(2 * np.pi) ** 2 * 2 * np.exp(-L * L / 2) / L
        assert abs(val - exact) / exact < 10 * tail + 1e-13
