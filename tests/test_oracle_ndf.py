"""Pins of the oracle's NDF integrator (Sec. 4.2, Eq. (ode_disc)): the printed
kappa_p and stability angles, the formula residual along a trajectory, the
order of convergence, the exact Rossby-Haurwitz evolution and the paper's
manufactured solution (Sec. 5, Example 1)."""
import math
import os

import numpy as np
import pytest

from oracle import layout
from oracle.ndf import NDF, Constants, rescale_matrix
from oracle.rhs import Problem, rhs_separable
from seeded_inputs import random_packed

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "ndf_coefficients.txt")


def _golden():
    rows = []
    with open(GOLDEN) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                p, k, a_ndf, a_bdf = line.split()
                rows.append((int(p), float(k), float(a_ndf), float(a_bdf)))
    return rows


def test_kappa_matches_paper():
    c = Constants()
    for p, kappa, _, _ in _golden():
        assert abs(c.kappa[p - 1] - kappa) < 1e-15


def _stability_angle(p, kappa):
    """A(alpha) angle of the constant-step NDFp/BDFp: boundary locus
    z(zeta) = sum_j (1/j)(1 - 1/zeta)^j - kappa gamma_p (1 - 1/zeta)^{p+1}
    on |zeta| = 1; alpha = smallest |arg(-z)| over the locus."""
    gamma = sum(1.0 / j for j in range(1, p + 1))
    t = np.linspace(1e-6, np.pi, 400001)
    w = 1.0 - np.exp(-1j * t)
    z = sum(w ** j / j for j in range(1, p + 1)) - kappa * gamma * w ** (p + 1)
    ang = np.abs(np.angle(-z))
    return math.degrees(float(np.min(ang)))


def test_stability_angles_match_paper():
    """The angles printed for NDF1..5 and for BDF3, BDF4 (Sec. 4.2); the
    paper prints whole degrees, truncated (BDF5's angle is 51.84 degrees)."""
    for p, kappa, a_ndf, a_bdf in _golden():
        got = min(_stability_angle(p, kappa), 90.0)
        assert a_ndf <= got + 1e-9 < a_ndf + 1.0, (p, got, a_ndf)
        got_bdf = min(_stability_angle(p, 0.0), 90.0)
        assert a_bdf <= got_bdf + 1e-9 < a_bdf + 1.0, (p, got_bdf, a_bdf)


def test_rescale_matrix_composition():
    """U^2 = I and R(r1)U R(r2)U = R(r1 r2)U (interpolation of the same
    polynomial), the identities behind the difference-array rescaling."""
    k = 5
    np.testing.assert_allclose(rescale_matrix(k, 1.0), np.eye(k), atol=1e-13)
    A = rescale_matrix(k, 0.7) @ rescale_matrix(k, 1.3)
    np.testing.assert_allclose(A, rescale_matrix(k, 0.91), atol=1e-12)


def _linear_problem(n=6, seed=0):
    rng = np.random.default_rng(seed)
    jd = -rng.uniform(0.5, 5.0, n) + 1j * rng.uniform(-2, 2, n)
    y0 = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    return jd, y0


def test_formula_residual_along_trajectory():
    """Each replayed step satisfies Eq. (ode_disc) at its order p on the
    stored history (constant h; backward history extended linearly as the
    initial difference D_0 = h F(y_0) implies)."""
    jd, y0 = _linear_problem()
    rhs = lambda t, y: jd * y
    h = 0.01
    nd = NDF(rhs, jd, 0.0, y0, rtol=1e-8, atol=1e-10, h0=h)
    c = Constants()
    f0 = rhs(0.0, y0)
    hist = [y0 - j * h * f0 for j in range(8, 0, -1)] + [y0.copy()]
    orders = [1, 1, 2, 2, 2, 3, 3, 3, 3, 4, 4, 4, 4, 4, 5, 5, 5, 5, 5, 5, 4, 3, 2, 1]
    for p in orders:
        nd.replay_step(h, p)
        hist.append(nd.y.copy())
        Y = np.array(hist[::-1])            # Y[0] = y_{n+1}, Y[1] = y_n, ...

        def nab(j):                          # nabla^j y_{n+1}
            return sum((-1) ** i * math.comb(j, i) * Y[i] for i in range(j + 1))
        lhs = sum(nab(j) / j for j in range(1, p + 1))
        res = lhs - h * rhs(0, Y[0]) - c.kappa[p - 1] * c.gamma[p - 1] * nab(p + 1)
        assert np.max(np.abs(res)) < 1e-13, (p, np.max(np.abs(res)))


@pytest.mark.parametrize("p", [1, 2, 3, 4, 5])
def test_order_of_convergence(p):
    """Fixed order p, exact starting differences: global error ~ h^p."""
    jd, y0 = _linear_problem(3, 1)
    jd = jd * 0.3
    T = 1.0
    errs = []
    for nsteps in (40, 80):
        h = T / nsteps
        nd = NDF(lambda t, y: jd * y, jd, 0.0, y0, rtol=1e-8, atol=1e-10, h0=h)
        ex = lambda t: y0 * np.exp(jd * t)
        hist = np.array([ex(-j * h) for j in range(p + 2)])
        for j in range(p + 1):
            nd.dif[j] = sum((-1) ** i * math.comb(j + 1, i) * hist[i] for i in range(j + 2))
        nd.k = p
        for _ in range(nsteps):
            nd.replay_step(h, p)
        errs.append(np.max(np.abs(nd.y - ex(T))))
    rate = math.log2(errs[0] / errs[1])
    assert abs(rate - p) < 0.35, (p, rate, errs)


def test_rossby_haurwitz_exact_evolution():
    """Single-degree data evolve as alpha(t) = alpha(0) exp((-nu lambda +
    2 i Omega m / lambda) t) (single-degree fields have B(u,u) a gradient);
    the adaptive oracle (oracle RHS) tracks it within the tolerance."""
    N, M = 8, 28
    prob = Problem(N, M, 2e-2, 1.0)
    a0 = np.where(prob.Ls == 4, random_packed(N, 2), 0)
    jd = -prob.nu * prob.lam + 2j * prob.Omega * prob.ms / prob.lam
    rtol = 1e-8
    nd = NDF(lambda t, y: rhs_separable(prob, y), jd, 0.0, a0, rtol=rtol,
             atol=1e-3 * rtol * np.max(np.abs(a0)), t_end=2.0)
    while nd.t < 2.0 - 1e-14:
        nd.step()
    exact = a0 * np.exp(jd * 2.0)
    assert np.max(np.abs(nd.y - exact)) <= 50 * rtol * np.max(np.abs(a0))


def _example1(prob, N0):
    """Exact coefficients of Sec. 5 Example 1 (Eqs. (g_for_ini), (exact_soln)):
    alpha(t) = t g(t) [L <= N0] + g(t) [L = 1] + (t - 1) g(t) [L = 2] on every
    packed (L, m >= 0) entry (2 Re Z_{L,m} = Z_{L,m} + (-1)^m Z_{L,-m} has
    packed coefficient 1), g(t) = nu e^{-t} (sin 5t + cos 10t)."""
    Ls = prob.Ls
    nu = prob.nu
    g = lambda t: nu * math.exp(-t) * (math.sin(5 * t) + math.cos(10 * t))
    dg = lambda t: nu * math.exp(-t) * (5 * math.cos(5 * t) - 10 * math.sin(10 * t)
                                        - math.sin(5 * t) - math.cos(10 * t))
    one = (Ls <= N0).astype(float)
    e1 = (Ls == 1).astype(float)
    e2 = (Ls == 2).astype(float)

    def alpha(t):
        return (t * g(t) * one + g(t) * e1 + (t - 1) * g(t) * e2).astype(complex)

    def dalpha(t):
        return ((g(t) + t * dg(t)) * one + dg(t) * e1 + (g(t) + (t - 1) * dg(t)) * e2).astype(complex)
    return alpha, dalpha


def test_manufactured_solution_example1():
    """Forcing chosen so that Example 1's field is the exact solution:
    fhat(t) = alpha'(t) + nu lambda alpha(t) + N(alpha(t)); the adaptive NDF
    run on the oracle RHS recovers alpha(T)."""
    N0 = 6
    prob = Problem(N0, 3 * N0 + 2, 1.0, 1.0)
    alpha, dalpha = _example1(prob, N0)
    nonlin = lambda a: -(rhs_separable(prob, a) + prob.nu * prob.lam * a)
    forcing = lambda t: dalpha(t) + prob.nu * prob.lam * alpha(t) + nonlin(alpha(t))
    rhs = lambda t, y: rhs_separable(prob, y, forcing(t))
    jd = -prob.nu * prob.lam + 2j * prob.Omega * prob.ms / prob.lam
    rtol = 1e-7
    T = 1.5
    nd = NDF(rhs, jd, 0.0, alpha(0.0), rtol=rtol, atol=1e-9, t_end=T)
    while nd.t < T - 1e-14:
        nd.step()
    err = np.linalg.norm(nd.y - alpha(T)) / np.linalg.norm(alpha(T))
    assert err < 1e-5, err
    s = layout.multiplicity(prob.ms)
    assert np.all(np.isfinite(s))


def test_adaptive_controller_changes_order_and_rejects():
    """The controller raises the order on a smooth problem and rejects a
    step that is far too large."""
    jd, y0 = _linear_problem(4, 3)
    nd = NDF(lambda t, y: jd * y, jd, 0.0, y0, rtol=1e-7, atol=1e-9, h0=1e-4)
    orders = [nd.step()["order"] for _ in range(60)]
    assert max(orders) >= 3
    nd.h = 5.0
    info = nd.step()
    assert info["rejections"] >= 1
