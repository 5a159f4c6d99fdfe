"""Pins of the oracle's quadrature (Eq. (quadrule)) and Legendre tables
(Eq. (sph_har)) against closed forms, exactness and library routines."""
import math

import numpy as np
import pytest

from oracle.legendre import (dtheta_from_degree_shift, dtheta_from_order_ladder,
                             pt_bruteforce, pt_table)
from oracle.quadrature import Grid, gauss_legendre


@pytest.mark.parametrize("n", [1, 4, 24, 48, 96, 384])
def test_gauss_exact_on_monomials(n):
    _, x, _, w = gauss_legendre(n)
    assert abs(w.sum() - 2.0) < 1e-14
    for k in range(0, 2 * n):
        exact = 0.0 if k % 2 else 2.0 / (k + 1)
        assert abs(np.sum(w * x ** k) - exact) < 2e-14 * max(1.0, exact) + 1e-15


@pytest.mark.parametrize("n", [5, 48, 100])
def test_gauss_matches_numpy_leggauss(n):
    _, x, _, w = gauss_legendre(n)
    xr, wr = np.polynomial.legendre.leggauss(n)
    order = np.argsort(-xr)
    np.testing.assert_allclose(x, xr[order], rtol=0, atol=2e-15)
    # numpy's weights carry ~1e-12 relative error near the poles (checked
    # against 40-digit mpmath weights); ours are checked by exactness above
    np.testing.assert_allclose(w, wr[order], rtol=5e-12)


def _sphere_monomial(a, b, c):
    """int_S x^a y^b z^c dS (closed form; zero unless all even)."""
    if a % 2 or b % 2 or c % 2:
        return 0.0
    g = math.gamma
    return 2.0 * g((a + 1) / 2) * g((b + 1) / 2) * g((c + 1) / 2) / g((a + b + c + 3) / 2)


@pytest.mark.parametrize("M", [8, 14])
def test_QM_exact_on_spherical_polynomials(M):
    """Q_M is exact on polynomials of degree <= M-1 (Sec. 3, below Eq. (quadrule))."""
    g = Grid(M)
    st = g.sin[:, None]
    X = st * np.cos(g.phi)[None, :]
    Y = st * np.sin(g.phi)[None, :]
    Z = np.repeat(g.x[:, None], M, axis=1)
    for a in range(M):
        for b in range(M - a):
            for c in range(M - a - b):
                val = g.integrate(X ** a * Y ** b * Z ** c)
                assert abs(val - _sphere_monomial(a, b, c)) < 1e-13


def test_QM_not_exact_beyond_degree():
    g = Grid(8)
    Z = np.repeat(g.x[:, None], 8, axis=1)
    assert abs(g.integrate(Z ** 8) - _sphere_monomial(0, 0, 8)) > 1e-6


def test_closed_form_low_degree():
    th = np.linspace(0.1, 3.0, 7)
    x, s = np.cos(th), np.sin(th)
    T = pt_table(2, x, s)
    pi = math.pi
    np.testing.assert_allclose(T[0][0], np.full_like(x, 1 / math.sqrt(4 * pi)), rtol=1e-15)
    np.testing.assert_allclose(T[0][1], math.sqrt(3 / (4 * pi)) * x, rtol=1e-14)
    np.testing.assert_allclose(T[1][0], -math.sqrt(3 / (8 * pi)) * s, rtol=1e-14)
    np.testing.assert_allclose(T[0][2], math.sqrt(5 / (16 * pi)) * (3 * x ** 2 - 1), rtol=1e-13, atol=1e-15)
    np.testing.assert_allclose(T[1][1], -math.sqrt(15 / (8 * pi)) * s * x, rtol=1e-13, atol=1e-15)
    np.testing.assert_allclose(T[2][0], math.sqrt(15 / (32 * pi)) * s ** 2, rtol=1e-14)
    for (L, m) in [(1, 0), (1, 1), (2, 0), (2, 1), (2, 2)]:
        np.testing.assert_allclose(pt_bruteforce(L, m, x, s), T[m][L - m], rtol=1e-13, atol=1e-15)


def test_recurrence_vs_bruteforce_and_scipy():
    _, x, s, _ = gauss_legendre(40)
    Lmax = 30
    T = pt_table(Lmax, x, s)
    for m in range(0, Lmax + 1, 3):
        for L in range(m, Lmax + 1, 2):
            ref = pt_bruteforce(L, m, x, s)
            np.testing.assert_allclose(T[m][L - m], ref, rtol=1e-11, atol=1e-13)
    sp = pytest.importorskip("scipy.special")
    if not hasattr(sp, "sph_harm_y"):
        pytest.skip("scipy without sph_harm_y")
    th = np.arccos(x)
    for (L, m) in [(3, 1), (10, 4), (25, 25), (30, 7)]:
        ref = sp.sph_harm_y(L, m, th, 0.0).real
        np.testing.assert_allclose(T[m][L - m], ref, rtol=1e-11, atol=1e-13)


@pytest.mark.parametrize("L,m", [(1, 0), (3, 2), (8, 0), (8, 5), (20, 11)])
def test_eigenfunction_of_laplacian(L, m):
    """-Delta Y = L(L+1) Y (Sec. 2, below Eq. (sph_har)), with the theta part
    checked by central differences of the tabulated function."""
    th = np.array([0.4, 0.9, 1.3, 2.2])
    h = 1e-3

    def P(t):
        return pt_table(L, np.cos(t), np.sin(t))[m][L - m]

    p0 = P(th)
    d1 = (P(th - 2 * h) - 8 * P(th - h) + 8 * P(th + h) - P(th + 2 * h)) / (12 * h)
    d2 = (-P(th - 2 * h) + 16 * P(th - h) - 30 * p0 + 16 * P(th + h) - P(th + 2 * h)) / (12 * h * h)
    lap = d2 + np.cos(th) / np.sin(th) * d1 - m * m / np.sin(th) ** 2 * p0
    np.testing.assert_allclose(lap, -L * (L + 1) * p0, atol=2e-7 * max(1.0, L * L))


def test_theta_derivative_three_ways():
    th = np.array([0.3, 1.0, 1.9, 2.7])
    x, s = np.cos(th), np.sin(th)
    Lmax = 15
    ext = pt_table(Lmax + 1, x, s)
    D = dtheta_from_degree_shift(ext, Lmax, s)
    h = 1e-5
    Tp = pt_table(Lmax, np.cos(th + h), np.sin(th + h))
    Tm = pt_table(Lmax, np.cos(th - h), np.sin(th - h))
    for m in range(Lmax + 1):
        for L in range(m, Lmax + 1):
            fd = (Tp[m][L - m] - Tm[m][L - m]) / (2 * h)
            lad = dtheta_from_order_ladder(L, m, x, s)
            np.testing.assert_allclose(D[m][L - m], lad, rtol=1e-11, atol=1e-12)
            np.testing.assert_allclose(D[m][L - m], fd, rtol=0, atol=2e-7 * L)


def test_orthonormality_by_quadrature():
    """(Y_{L,m}, Y_{L',m}) = delta (Eq. (sph_har), orthonormal basis), exact
    under Q_M for L + L' <= M - 1."""
    M = 24
    g = Grid(M)
    Lmax = 11
    T = pt_table(Lmax, g.x, g.sin)
    for m in range(Lmax + 1):
        P = T[m]
        G = 2 * np.pi * (P * g.w[None, :]) @ P.T   # phi integral of |e^{im phi}|^2 = 2 pi
        np.testing.assert_allclose(G, np.eye(P.shape[0]), atol=1e-14)


def _pt_mpmath(mp, L, m, t):
    """Pt_L^m(cos t) in 60-digit arithmetic by the unnormalised recurrence
    (K-m) P_K^m = (2K-1) x P_{K-1}^m - (K+m-1) P_{K-2}^m from
    P_m^m = (-1)^m (2m-1)!! sin^m and the factorial normalisation of
    Eq. (sph_har); mpmath's exponent range is unbounded."""
    mp.mp.dps = 60
    x, s = mp.cos(mp.mpf(t)), mp.sin(mp.mpf(t))
    pmm = (-1) ** m * mp.fac2(2 * m - 1) * s ** m
    p_prev, p = mp.mpf(0), pmm
    for K in range(m + 1, L + 1):
        p_prev, p = p, ((2 * K - 1) * x * p - (K + m - 1) * p_prev) / (K - m)
    return mp.sqrt((2 * L + 1) / (4 * mp.pi) * mp.factorial(L - m) / mp.factorial(L + m)) * p


def test_extended_exponent_at_high_order():
    """Near the pole at L = 511 the diagonal sin^m underflows binary64; the
    extended exponent must keep the values that are representable."""
    mp = pytest.importorskip("mpmath")
    th = np.array([0.05, 0.3, 1.2])
    x, s = np.cos(th), np.sin(th)
    Lmax = 512
    T = pt_table(Lmax, x, s)
    checked = 0
    for (L, m) in [(512, 200), (512, 400), (300, 290), (511, 100), (512, 30), (450, 449)]:
        for i, t in enumerate(th):
            ref = float(_pt_mpmath(mp, L, m, t))
            got = T[m][L - m][i]
            if abs(ref) > 1e-290:
                assert abs(got - ref) <= 1e-12 * abs(ref), (L, m, t, got, ref)
                checked += 1
            else:
                assert abs(got) < 1e-280
    assert checked >= 8
    assert np.all(np.isfinite(np.concatenate([t.ravel() for t in T])))
