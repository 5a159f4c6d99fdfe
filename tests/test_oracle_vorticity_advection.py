"""Independent pins of the vorticity zeta and of the nonlinear term.

The oracle writes zeta = sum lambda_L^{1/2} alpha_{L,m} Y_{L,m} (Eq. (vort_app))
and the nonlinear term as ((zeta + 2 Omega cos theta) xhat x u, Z_{L,m})_M
(Eqs. (short_nonlin1), (C)).  The invariants and the single-degree closed form
hold for any constant multiple of zeta, so these tests reach both from the
velocity u alone, by routes that use neither formula:

* zeta from its definition Curl_n u = -xhat Div(xhat x u) (Eq. (Curl)): the
  surface divergence is the trace of the tangential derivative, taken by a
  sixth-order central difference along two orthogonal great circles through
  each node of the embedded unit sphere;
* zeta through the duality (Curl psi, v) = (psi, Curl_n v) of
  Eq. (ip_identities1): (zeta, Y_{L,m}) = (u, Curl Y_{L,m}), with
  Curl Y = -xhat x Grad Y formed as a Cartesian cross product;
* the covariant derivative grad_u u of the Navier-Stokes system
  (Eq. (NSE_sphere)), taken as the tangential part of the derivative of the
  Cartesian velocity along the great circle with initial velocity u (the
  Levi-Civita connection of a surface in R^3).  Pointwise, grad_u u minus the
  finite-difference Grad(|u|^2/2) must equal zeta xhat x u (Eq.
  (short_nonlin1)); projected on Z_{L,m} with the Coriolis field of Eq. (C)
  it must give the oracle's nonlinear term.

The velocity at an arbitrary point is u = sum alpha lambda^{-1/2} Curl Y with
Grad Y = d_theta Y e_theta + (1/sin theta) d_phi Y e_phi (textbook surface
gradient) and Y from the brute-force Legendre routine, both pinned elsewhere
against scipy and closed forms.  Planted mistakes zeta -> -zeta and
zeta -> 2 zeta in the oracle are each caught.
"""
import numpy as np
import pytest

import oracle.rhs as R
from oracle import layout
from oracle.legendre import dtheta_from_order_ladder, pt_bruteforce_signed
from oracle.rhs import Problem, project_scalar, rhs_separable, synthesize
from seeded_inputs import random_packed

# sixth-order central first derivative, offsets -3..3 (steps of h)
_FD = np.array([-1.0, 9.0, -45.0, 0.0, 45.0, -9.0, 1.0]) / 60.0
_OFF = np.arange(-3, 4)
_H = 4e-3


def _angles(X):
    theta = np.arccos(np.clip(X[..., 2], -1.0, 1.0))
    phi = np.arctan2(X[..., 1], X[..., 0])
    return theta, phi


def _frame(theta, phi):
    """Cartesian xhat, e_theta, e_phi."""
    st, ct, sp, cp = np.sin(theta), np.cos(theta), np.sin(phi), np.cos(phi)
    xh = np.stack([st * cp, st * sp, ct], -1)
    et = np.stack([ct * cp, ct * sp, -st], -1)
    ep = np.stack([-sp, cp, np.zeros_like(sp)], -1)
    return xh, et, ep


def _grad_Y(L, m, X):
    """Complex Cartesian Grad Y_{L,m} at unit vectors X (..., 3), and Y."""
    theta, phi = _angles(X)
    x, s = np.cos(theta), np.sin(theta)
    e = np.exp(1j * m * phi)
    Y = pt_bruteforce_signed(L, m, x, s) * e
    dY = dtheta_from_order_ladder(L, m, x, s) * e
    _, et, ep = _frame(theta, phi)
    return dY[..., None] * et + (1j * m * Y / s)[..., None] * ep, Y


def _velocity(full, X):
    """Real Cartesian u = sum alpha lambda^{-1/2} (-xhat x Grad Y) at X."""
    u = np.zeros(X.shape, dtype=np.complex128)
    for (L, m), a in full.items():
        G, _ = _grad_Y(L, m, X)
        u += a / np.sqrt(L * (L + 1.0)) * np.cross(-X, G)
    assert np.max(np.abs(u.imag)) < 1e-12 * (1.0 + np.max(np.abs(u.real)))
    return u.real


def _unit(V):
    n = np.linalg.norm(V, axis=-1, keepdims=True)
    return np.where(n > 0, V / np.where(n > 0, n, 1.0), 0.0), n


def _along(F, X, V):
    """d/ds F(gamma(s)) at s = 0 on the great circle through X with
    gamma'(0) = V: |V| times the arc-length derivative along V/|V|, taken at
    the arc-length points cos(o h) X + sin(o h) V/|V|."""
    d, n = _unit(V)
    acc = sum(c * F(np.cos(o * _H) * X + np.sin(o * _H) * d)
              for c, o in zip(_FD, _OFF) if c) / _H
    return acc * (n if acc.ndim == n.ndim else n[..., 0])


def _nodes(prob):
    g = prob.grid
    th = np.repeat(g.theta[:, None], g.M, axis=1)
    ph = np.repeat(g.phi[None, :], g.nlat, axis=0)
    return th, ph


def _zeta_by_divergence(prob, full):
    """zeta = -Div(xhat x u) at the nodes (Eq. (Curl)), Div by the trace of
    the tangential derivative."""
    th, ph = _nodes(prob)
    X, et, ep = _frame(th, ph)

    def V(P):
        return np.cross(P, _velocity(full, P))
    div = sum(np.sum(t * _along(V, X, t), axis=-1) for t in (et, ep))
    return -div


def _advection(prob, full):
    """grad_u u and Grad(|u|^2/2) at the nodes, Cartesian."""
    th, ph = _nodes(prob)
    X, et, ep = _frame(th, ph)
    u = _velocity(full, X)
    D = _along(lambda P: _velocity(full, P), X, u)
    cov = D - np.sum(X * D, axis=-1, keepdims=True) * X

    def ke(P):
        v = _velocity(full, P)
        return 0.5 * np.sum(v * v, axis=-1)
    grad_ke = sum(_along(ke, X, t)[..., None] * t for t in (et, ep))
    return X, u, cov, grad_ke


def _state(N, seed):
    a = random_packed(N, seed)
    return a, layout.full_from_packed(a, N)


def zeta_defect(prob, a, full):
    z_or, _, _ = synthesize(prob, a)
    z_fd = _zeta_by_divergence(prob, full)
    return np.max(np.abs(z_or - z_fd)) / np.max(np.abs(z_fd))


def duality_defect(prob, a, full):
    """|(zeta, Y_{L,m})_M - (u, Curl Y_{L,m})_M| over every packed (L, m)."""
    z_or, _, _ = synthesize(prob, a)
    lhs = project_scalar(prob, z_or)
    th, ph = _nodes(prob)
    X, _, _ = _frame(th, ph)
    u = _velocity(full, X)
    wq = (2.0 * np.pi / prob.M) * prob.grid.w[:, None]
    rhs = np.empty_like(lhs)
    for i, (L, m) in enumerate(zip(prob.Ls, prob.ms)):
        G, _ = _grad_Y(int(L), int(m), X)
        curlY = np.cross(-X, G)
        rhs[i] = np.sum(wq * np.sum(u * np.conj(curlY), axis=-1))
    return np.max(np.abs(lhs - rhs)) / np.max(np.abs(rhs))


def lamb_defect(prob, a, full):
    """Pointwise grad_u u - Grad(|u|^2/2) against the oracle's zeta xhat x u."""
    X, u, cov, grad_ke = _advection(prob, full)
    z_or, _, _ = synthesize(prob, a)
    lamb = z_or[..., None] * np.cross(X, u)
    return np.max(np.abs(cov - grad_ke - lamb)) / np.max(np.abs(lamb))


def nonlinear_defect(prob, a, full):
    """(grad_u u + C u, Z_{L,m})_M against the oracle's nonlinear term."""
    X, u, cov, _ = _advection(prob, full)
    th, _ = _nodes(prob)
    W = cov + (2.0 * prob.Omega * np.cos(th))[..., None] * np.cross(X, u)
    wq = (2.0 * np.pi / prob.M) * prob.grid.w[:, None]
    Nfd = np.empty(prob.n(), dtype=np.complex128)
    for i, (L, m) in enumerate(zip(prob.Ls, prob.ms)):
        G, _ = _grad_Y(int(L), int(m), X)
        Z = np.cross(-X, G) / np.sqrt(L * (L + 1.0))
        Nfd[i] = np.sum(wq * np.sum(W * np.conj(Z), axis=-1))
    Nor = -(rhs_separable(prob, a) + prob.nu * prob.lam * a)
    return np.linalg.norm(Nor - Nfd) / np.linalg.norm(Nfd)


@pytest.mark.parametrize("N,M,seed", [(3, 12, 31), (5, 18, 32), (6, 22, 33)])
def test_vorticity_is_curl_n_of_velocity(N, M, seed):
    prob = Problem(N, M, 1e-2, 1.0)
    a, full = _state(N, seed)
    assert zeta_defect(prob, a, full) < 1e-9


@pytest.mark.parametrize("N,M,seed", [(4, 14, 41), (6, 20, 42)])
def test_vorticity_duality_with_curl(N, M, seed):
    prob = Problem(N, M, 1e-2, 1.0)
    a, full = _state(N, seed)
    assert duality_defect(prob, a, full) < 1e-13


@pytest.mark.parametrize("N,M,seed", [(3, 12, 51), (5, 18, 52)])
def test_lamb_vector_form_of_advection(N, M, seed):
    """grad_u u = Grad(|u|^2/2) + zeta xhat x u pointwise (Eq. (short_nonlin1))."""
    prob = Problem(N, M, 1e-2, 1.0)
    a, full = _state(N, seed)
    assert lamb_defect(prob, a, full) < 1e-9


@pytest.mark.parametrize("N,M,Omega,seed", [(3, 12, 0.0, 61), (5, 18, 1.7, 62),
                                             (6, 20, 0.4, 63)])
def test_nonlinear_term_from_covariant_derivative(N, M, Omega, seed):
    """The oracle's projected nonlinear plus Coriolis term equals the
    projection of grad_u u + C u obtained without the zeta formula."""
    prob = Problem(N, M, 3e-3, Omega)
    a, full = _state(N, seed)
    assert nonlinear_defect(prob, a, full) < 1e-9


def test_triad_formula_of_eval_nonlin1_with_sign_reading():
    """Eq. (eval_nonlin1) gives the nonlinear term mode by mode:
    (B(Z_R, Z_J), Z_L) = c sqrt(lambda_R/(lambda_J lambda_L))
    (Y_R Grad Y_J, xhat x Grad Y_L).  It is printed with c = +1, but
    Eq. (eval_nonlin), Z = lambda^{-1/2} Curl Y and Curl Y = -xhat x Grad Y
    (Eqs. (stok_eig), (Curl)) give c = -1, and the covariant-derivative pin
    above agrees with c = -1.  Reading: c = -1.  Summed over all triads of a
    random state at Omega = 0 it reproduces the oracle's nonlinear term."""
    N, M = 4, 16
    prob = Problem(N, M, 0.0, 0.0)
    a, full = _state(N, 81)
    th, ph = _nodes(prob)
    X, _, _ = _frame(th, ph)
    wq = (2.0 * np.pi / M) * prob.grid.w[:, None]
    modes = {k: _grad_Y(k[0], k[1], X) for k in full}
    # sum_R alpha_R lambda_R^{1/2} Y_R and sum_J alpha_J lambda_J^{-1/2} Grad Y_J
    zY = sum(full[k] * np.sqrt(k[0] * (k[0] + 1.0)) * modes[k][1] for k in full)
    gJ = sum(full[k] / np.sqrt(k[0] * (k[0] + 1.0)) * modes[k][0] for k in full)
    triad = np.empty(prob.n(), dtype=np.complex128)
    for i, (L, m) in enumerate(zip(prob.Ls, prob.ms)):
        GL = modes[(int(L), int(m))][0]
        xg = np.cross(X, GL) / np.sqrt(L * (L + 1.0))
        triad[i] = np.sum(wq * np.sum(zY[..., None] * gJ * np.conj(xg), axis=-1))
    Nor = -rhs_separable(prob, a)
    assert np.linalg.norm(Nor + triad) <= 1e-13 * np.linalg.norm(Nor)
    assert np.linalg.norm(Nor - triad) > np.linalg.norm(Nor)


# ---------------------------------------------------------------------------
# planted mistakes in the oracle's vorticity: each pin above must catch them

def _plant_zeta_scale(monkeypatch, c):
    good = R.spectral_fields

    def wrong(prob, alpha):
        z, ut, up = good(prob, alpha)
        return c * z, ut, up
    monkeypatch.setattr(R, "spectral_fields", wrong)


@pytest.mark.parametrize("c", [-1.0, 2.0])
def test_planted_mistake_zeta_scale_is_caught(monkeypatch, c):
    _plant_zeta_scale(monkeypatch, c)
    N, M = 4, 14
    prob = Problem(N, M, 3e-3, 0.9)
    a, full = _state(N, 71)
    assert zeta_defect(prob, a, full) > 0.3
    assert duality_defect(prob, a, full) > 0.3
    assert lamb_defect(prob, a, full) > 0.3
    assert nonlinear_defect(prob, a, full) > 0.1


def test_planted_mistake_zeta_sign_survives_invariants(monkeypatch):
    """Why the pins above are needed: with zeta -> -zeta the energy and
    enstrophy invariants and the single-degree closed form still hold."""
    _plant_zeta_scale(monkeypatch, -1.0)
    N, M = 6, 20
    prob = Problem(N, M, 1e-3, 1.3)
    a = random_packed(N, 72)
    Nw = -(R.rhs_separable(prob, a) + prob.nu * prob.lam * a)
    s = layout.multiplicity(prob.ms)
    e = np.sum(s * np.conj(a) * Nw).real / (np.linalg.norm(a) * np.linalg.norm(Nw))
    z = np.sum(s * prob.lam * np.conj(a) * Nw).real / (
        np.linalg.norm(prob.lam * a) * np.linalg.norm(Nw))
    assert abs(e) < 1e-13 and abs(z) < 1e-13
    one = np.where(prob.Ls == 3, a, 0)
    F = R.rhs_separable(prob, one)
    expect = (-prob.nu * prob.lam + 2j * prob.Omega * prob.ms / prob.lam) * one
    assert np.linalg.norm(F - expect) <= 1e-13 * np.linalg.norm(expect)
