"""Pins of the oracle's diagnostics (Sec. 6.2): the energy spectrum of
Eq. (energy) against Parseval sums of the synthesised field on the grid and
per degree through the brute-force basis, truncation and resizing, and the
approximate inertial manifold of Eq. (eq:p-p) against (i) the vanishing
nonlinear term of single-degree fields, (ii) the linearised RHS at rest (its
band modes are the steady state of du/dt = f - (nu A + C) u), (iii) a
brute-force evaluation of B.  The last test plants a mistake in the oracle."""
import numpy as np
import pytest

import oracle.diagnostics as D
from oracle import layout
from oracle.rhs import Problem, basis_bruteforce, rhs_bruteforce, synthesize
from oracle.tlm import rhs_tlm
from seeded_inputs import coefficients


@pytest.mark.parametrize("N,M", [(5, 18), (12, 38)])
def test_energy_spectrum_parseval(N, M):
    """sum_L E(L) = Q_M(|u|^2): Z is orthonormal and |u|^2 has degree 2N <= M - 1."""
    prob = Problem(N, M, 1e-2, 1.0)
    a = coefficients(N, 31 + N, 0.1)
    _, uth, uph = synthesize(prob, a)
    energy = prob.grid.integrate(uth ** 2 + uph ** 2)
    E = D.energy_spectrum(N, a)
    assert E[0] == 0.0
    assert abs(E.sum() - energy) <= 1e-13 * energy


def test_energy_per_degree_bruteforce():
    """E(L) = Q_M(|u_L|^2) with u_L the degree-L part summed from every basis
    field Z_{L,m} at every node (all signed orders)."""
    N, M = 4, 16
    prob = Problem(N, M, 1e-2, 1.0)
    a = coefficients(N, 77, 0.05)
    basis = basis_bruteforce(prob)
    full = layout.full_from_packed(a, N)
    E = D.energy_spectrum(N, a)
    for L in range(1, N + 1):
        ut = sum(full[(L, m)] * basis[(L, m)][1] for m in range(-L, L + 1))
        up = sum(full[(L, m)] * basis[(L, m)][2] for m in range(-L, L + 1))
        eL = prob.grid.integrate(np.abs(ut) ** 2 + np.abs(up) ** 2)
        assert abs(E[L] - eL) <= 1e-13 * max(eL, 1e-300), L


def test_truncate_and_resize():
    N, N2 = 9, 14
    a = coefficients(N, 5, 0.1)
    b = D.resize(N, a, N2)
    np.testing.assert_array_equal(D.resize(N2, b, N), a)
    Ls, _ = layout.packed_degrees_orders(N2)
    assert np.all(b[Ls > N] == 0)
    np.testing.assert_array_equal(D.resize(N, a, 6), D.resize(N, D.truncate(N, a, 6), 6))
    E = D.energy_spectrum(N2, b)
    np.testing.assert_allclose(E[: N + 1], D.energy_spectrum(N, a), rtol=0, atol=0)


def test_inertial_manifold_single_degree_is_zero():
    """A single-degree field (all modes on one degree J <= N1) has B(u, u) a
    gradient (Eq. (short_nonlin1) with zeta = lambda_J psi), so without forcing
    Phi(u) = 0."""
    N1, N2, M = 4, 8, 26
    prob = Problem(N2, M, 1e-2, 1.7)
    a = D.resize(N1, coefficients(N1, 9, 0.0), N2)
    Ls, _ = layout.packed_degrees_orders(N2)
    a = np.where(Ls == 3, a, 0.0)
    phi = D.inertial_manifold(prob, N1, a)
    assert np.max(np.abs(phi)) <= 1e-14 * np.max(np.abs(a))


def test_inertial_manifold_at_rest_is_linear_steady_state():
    """u1 = 0: Phi's band modes solve f - (nu A + C) Phi = 0, with (nu A + C)
    applied through the linearised RHS at rest (transforms and the grid
    product 2 Omega cos(theta) xhat x u, not the diagonal formula)."""
    N1, N2, M = 3, 7, 24
    prob = Problem(N2, M, 3e-2, 1.3)
    f = coefficients(N2, 21, 0.0)
    phi = D.inertial_manifold(prob, N1, np.zeros_like(f), f)
    r = f + rhs_tlm(prob, np.zeros_like(f), phi)
    band = prob.Ls > N1
    assert np.max(np.abs(r[band])) <= 1e-13 * np.max(np.abs(f))
    assert np.all(phi[~band] == 0)


def test_inertial_manifold_bruteforce_B():
    """f - B(u1, u1) on the band from the brute-force RHS (every Z at every
    node) gives the same Phi."""
    N1, N2, M = 3, 6, 20
    prob = Problem(N2, M, 1e-2, 0.9)
    a = D.resize(N1, coefficients(N1, 41, 0.1) * 5, N2)
    f = coefficients(N2, 42, 0.2)
    phi = D.inertial_manifold(prob, N1, a, f)
    Fb = rhs_bruteforce(prob, a, f)
    band = prob.Ls > N1
    res = prob.nu * prob.lam - 2j * prob.Omega * prob.ms / prob.lam
    np.testing.assert_allclose(phi[band] * res[band], Fb[band], rtol=0, atol=1e-13 * np.max(np.abs(Fb)))


def test_planted_mistake_resolvent_sign(monkeypatch):
    """(nu A - C) instead of (nu A + C) in the oracle is caught by the
    linear steady-state pin."""
    orig = D.inertial_manifold

    def wrong(prob, N1, alpha, forcing=None):
        phi = orig(prob, N1, alpha, forcing)
        good = prob.nu * prob.lam - 2j * prob.Omega * prob.ms / prob.lam
        bad = prob.nu * prob.lam + 2j * prob.Omega * prob.ms / prob.lam
        return phi * good / bad

    monkeypatch.setattr(D, "inertial_manifold", wrong)
    with pytest.raises(AssertionError):
        test_inertial_manifold_at_rest_is_linear_steady_state()
