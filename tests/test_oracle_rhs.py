"""Pins of the oracle's RHS F (Eq. (ode)) against what the paper and the
mathematics fix: orthonormality of Z (Eq. (Fourier_coeff)), transform round
trips (Eq. (disc_proj_prop1)), the discrete invariants of Thm 4.1, the
diagonal Coriolis identity Eq. (Coriolis_ZLm), single-degree (Rossby-Haurwitz)
fields, Hermitian symmetry, and brute force vs separable evaluation.  The last
tests plant mistakes in the oracle and check that a pin catches each."""
import numpy as np
import pytest

import oracle.rhs as R
from oracle import layout
from oracle.rhs import (Problem, basis_bruteforce, project, project_scalar,
                        rhs_bruteforce, rhs_separable, synthesize)
from oracle.tlm import rhs_tlm
from seeded_inputs import coefficients, random_packed


def _energy_pair(prob, a, N):
    s = layout.multiplicity(prob.ms)
    e = np.sum(s * (np.conj(a) * N)).real
    z = np.sum(s * prob.lam * (np.conj(a) * N)).real
    return (e / (np.linalg.norm(a) * np.linalg.norm(N)),
            z / (np.linalg.norm(prob.lam * a) * np.linalg.norm(N)))


def _nonlinear(prob, a, F=None):
    F = rhs_separable(prob, a) if F is None else F
    return -(F + prob.nu * prob.lam * a)


@pytest.mark.parametrize("N,M", [(3, 12), (7, 24), (12, 38)])
def test_bruteforce_vs_separable(N, M):
    prob = Problem(N, M, 1e-2, 1.3)
    a = random_packed(N, 11)
    f = random_packed(N, 12, 0.1)
    Fb, info = rhs_bruteforce(prob, a, f, return_all=True)
    Fs = rhs_separable(prob, a, f)
    assert np.linalg.norm(Fb - Fs) <= 1e-13 * np.linalg.norm(Fb)
    assert info["imag"] < 1e-12
    # Hermitian symmetry N_{L,-m} = (-1)^m conj N_{L,m}
    Nf = info["N"]
    for (L, m), v in Nf.items():
        if m > 0:
            assert abs(Nf[(L, -m)] - (-1) ** m * np.conj(v)) <= 1e-13 * (1 + abs(v))


def test_bruteforce_vs_separable_L31_grid():
    """The L = 31, 48 x 96 workload grid."""
    prob = Problem(31, 96, 1e-2, 1.0)
    a = coefficients(31, 1, 0.3)
    Fb = rhs_bruteforce(prob, a)
    Fs = rhs_separable(prob, a)
    assert np.linalg.norm(Fb - Fs) <= 1e-13 * np.linalg.norm(Fb)


def test_Z_orthonormal_and_curl_free_orthogonal():
    """(Z_{L,m}, Z_{L',m'})_M = delta and (Z_{L,m}, Grad Y_{L',m'})_M = 0 for
    degrees that Q_M integrates exactly (Sec. 2, Hodge decomposition)."""
    N, M = 5, 14
    prob = Problem(N, M, 1.0, 1.0)
    B = basis_bruteforce(prob)
    g = prob.grid
    wq = (2 * np.pi / M) * g.w[:, None]
    keys = list(B)
    G = np.zeros((len(keys), len(keys)), dtype=complex)
    H = np.zeros_like(G)
    for i, ki in enumerate(keys):
        _, Zt, Zp = B[ki]
        for j, kj in enumerate(keys):
            Y, Ut, Up = B[kj]
            G[i, j] = np.sum(wq * (Zt * np.conj(Ut) + Zp * np.conj(Up)))
            # Grad Y_{L',m'} = -xhat x Curl Y ... in components: (d_theta Y, i m Y / sin)
            L2 = kj[0]
            gt = -Up * np.sqrt(L2 * (L2 + 1.0))        # d_theta Y
            gp = Ut * np.sqrt(L2 * (L2 + 1.0))          # i m Y / sin
            H[i, j] = np.sum(wq * (Zt * np.conj(gt) + Zp * np.conj(gp)))
    np.testing.assert_allclose(G, np.eye(len(keys)), atol=1e-13)
    np.testing.assert_allclose(H, 0, atol=1e-13)


@pytest.mark.parametrize("N,M", [(7, 24), (16, 52), (31, 96)])
def test_round_trip(N, M):
    """Discrete projection of a field of V_N returns its coefficients
    (Eq. (disc_proj_prop1)); the scalar analogue for zeta."""
    prob = Problem(N, M, 1.0, 1.0)
    a = random_packed(N, 5)
    z, ut, up = synthesize(prob, a)
    assert np.linalg.norm(project(prob, ut, up) - a) <= 1e-13 * np.linalg.norm(a)
    assert np.linalg.norm(project_scalar(prob, z) - np.sqrt(prob.lam) * a) \
        <= 1e-13 * np.linalg.norm(np.sqrt(prob.lam) * a)


@pytest.mark.parametrize("N,M", [(7, 24), (31, 96), (40, 124)])
def test_energy_and_enstrophy_invariants(N, M):
    """(B(u,u) + C u, u)_M = 0 and (B(u,u) + C u, A u)_M = 0 (Thm 4.1 and
    Eqs. (CuNuN), (CuNAuN))."""
    prob = Problem(N, M, 1e-3, 2.0)
    a = coefficients(N, 3, 0.05)
    e, z = _energy_pair(prob, a, _nonlinear(prob, a))
    assert abs(e) < 1e-13
    assert abs(z) < 1e-13


def test_enstrophy_invariant_needs_exact_quadrature():
    """With M below 3N + 2 (Eq. (M_choice)) the enstrophy invariant fails;
    the energy invariant holds pointwise for any M."""
    N = 12
    a = random_packed(N, 9)
    prob = Problem(N, 2 * N + 2, 1e-3, 1.0)
    e, z = _energy_pair(prob, a, _nonlinear(prob, a))
    assert abs(e) < 1e-13
    assert abs(z) > 1e-4


@pytest.mark.parametrize("N,M1,M2", [(12, 38, 48), (31, 96, 128), (5, 18, 64)])
def test_rhs_is_the_same_on_every_exact_grid(N, M1, M2):
    """Any even M >= 3N + 2 integrates the Galerkin terms exactly (Eq.
    (M_choice)), so F does not depend on the grid beyond rounding; below the
    bound it does."""
    a = random_packed(N, 21)
    F1 = rhs_separable(Problem(N, M1, 1e-3, 1.0), a)
    F2 = rhs_separable(Problem(N, M2, 1e-3, 1.0), a)
    assert np.linalg.norm(F1 - F2) <= 1e-13 * np.linalg.norm(F1)
    F0 = rhs_separable(Problem(N, 2 * N + 2, 1e-3, 1.0), a)
    assert np.linalg.norm(F0 - F1) > 1e-6 * np.linalg.norm(F1)


@pytest.mark.parametrize("L", [1, 4, 9])
def test_single_degree_rossby_haurwitz(L):
    """All coefficients on one degree: B(u,u) is a gradient, so only the
    diagonal terms survive, F = (-nu lambda + 2 i Omega m / lambda) alpha
    (Eqs. (eval_nonlin), (Coriolis_ZLm))."""
    N, M = 10, 34
    prob = Problem(N, M, 3e-3, 1.7)
    a = np.where(prob.Ls == L, random_packed(N, 21), 0)
    F = rhs_separable(prob, a)
    expect = (-prob.nu * prob.lam + 2j * prob.Omega * prob.ms / prob.lam) * a
    assert np.linalg.norm(F - expect) <= 1e-13 * np.linalg.norm(expect)


def test_coriolis_operator_is_diagonal():
    """Linear part of F at alpha = 0: (C Z_{J,k}, Z_{L,m}) = -2 Omega i m /
    lambda_L delta (Eq. (Coriolis_ZLm) with Z = lambda^{-1/2} Curl Y)."""
    N, M = 5, 18
    prob = Problem(N, M, 0.0, 1.9)
    n = prob.n()
    zero = np.zeros(n, dtype=complex)
    for j in range(n):
        for unit in (1.0, 1j):
            e = np.zeros(n, dtype=complex)
            e[j] = unit
            if prob.ms[j] == 0 and unit == 1j:
                continue
            col = rhs_tlm(prob, zero, e)
            expect = np.zeros(n, dtype=complex)
            expect[j] = 2j * prob.Omega * prob.ms[j] / prob.lam[j] * unit
            np.testing.assert_allclose(col, expect, atol=1e-14)


def test_split_coriolis_equals_full_rhs():
    """The split variant (Coriolis as its diagonal, Eq. (Coriolis_ZLm), and a
    product without 2 Omega cos(theta)) gives the same F at a nonlinear
    state: F_Omega(alpha) = F_0(alpha) + 2 i Omega m / lambda alpha."""
    N, M = 12, 38
    a = coefficients(N, 91, 0.2) * 3.0
    full = rhs_separable(Problem(N, M, 1e-2, 2.3), a)
    prob0 = Problem(N, M, 1e-2, 0.0)
    split = rhs_separable(prob0, a) + 2j * 2.3 * prob0.ms / prob0.lam * a
    np.testing.assert_allclose(split, full, atol=1e-13 * np.abs(full).max())


@pytest.mark.parametrize("N,M,Omega", [(12, 38, 0.0), (31, 96, 1.3)])
def test_advection_has_no_degree_one_component(N, M, Omega):
    """The advection term conserves the flow's angular momentum, whose
    components are the degree-1 coefficients (Z_{1,m} = lambda_1^{-1/2}
    Curl Y_{1,m} are the solid-body rotations): (B(u,u), Z_{1,m}) = 0 for any
    u.  At L = 1 only the Coriolis diagonal of Eq. (Coriolis_ZLm) remains."""
    prob = Problem(N, M, 1e-3, Omega)
    a = random_packed(N, 77)
    Nn = _nonlinear(prob, a)
    cor = -2j * Omega * prob.ms / prob.lam * a
    one = prob.Ls == 1
    assert np.linalg.norm((Nn - cor)[one]) <= 1e-14 * np.linalg.norm(Nn)
    assert np.linalg.norm(Nn[prob.Ls == 2]) > 1e-3 * np.linalg.norm(Nn)


# ---------------------------------------------------------------------------
# planted mistakes: each must be caught by one of the pins above

def test_planted_mistake_coriolis_sign(monkeypatch):
    def wrong(prob, zeta, uth, uph):
        q = zeta - 2.0 * prob.Omega * prob.grid.x[:, None]
        return -q * uph, q * uth
    monkeypatch.setattr(R, "pointwise_product", wrong)
    N, M = 6, 22
    prob = Problem(N, M, 0.0, 1.0)
    a = np.where(prob.Ls == 3, random_packed(N, 4), 0)
    F = R.rhs_separable(prob, a)
    expect = 2j * prob.Omega * prob.ms / prob.lam * a
    assert np.linalg.norm(F - expect) > 1e-3 * np.linalg.norm(expect)


def test_planted_mistake_dropped_degree_shift_term(monkeypatch):
    """Dropping the (L+1) eps_{L,m} Pt_{L-1} term of the theta derivative
    breaks brute force vs separable agreement and the round trip."""
    import oracle.legendre as LG

    def wrong(table_ext, Lmax, s):
        out = []
        for m in range(Lmax + 1):
            Tm = table_ext[m]
            d = np.empty((Lmax - m + 1, Tm.shape[1]))
            for L in range(m, Lmax + 1):
                d[L - m] = L * float(LG.eps(L + 1, m)) * Tm[L + 1 - m] / s
            out.append(d)
        return out
    monkeypatch.setattr(R, "dtheta_from_degree_shift", wrong)
    prob = Problem(5, 18, 1e-2, 1.0)
    a = random_packed(5, 3)
    Fb = rhs_bruteforce(prob, a)
    Fs = R.rhs_separable(prob, a)
    assert np.linalg.norm(Fb - Fs) > 1e-3 * np.linalg.norm(Fb)


def test_planted_mistake_swapped_product_components(monkeypatch):
    """W = q xhat x u with components swapped (a transposed operand) breaks
    the energy invariant."""
    def wrong(prob, zeta, uth, uph):
        q = zeta + 2.0 * prob.Omega * prob.grid.x[:, None]
        return q * uth, -q * uph
    monkeypatch.setattr(R, "pointwise_product", wrong)
    prob = Problem(7, 24, 1e-3, 1.0)
    a = random_packed(7, 8)
    N = -(R.rhs_separable(prob, a) + prob.nu * prob.lam * a)
    e, _ = _energy_pair(prob, a, N)
    assert abs(e) > 1e-3
