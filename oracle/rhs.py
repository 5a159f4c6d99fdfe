"""Right-hand side F(t, alpha) of the ODE system Eq. (ode).  Oracle only.

For alpha in V_N (Eq. (fin_space_vec)) and L = 1..N, |m| <= L:

  F_{L,m} = fhat_{L,m} - nu lambda_L alpha_{L,m}
            - ( (zeta + 2 Omega cos theta) xhat x u , Z_{L,m} )_M

* u = sum alpha_{L,m} Z_{L,m} (Eq. (app_soln_rep)),
  Z_{L,m} = lambda_L^{-1/2} Curl Y_{L,m}, Curl v = -xhat x Grad v,
  lambda_L = L(L+1) (Eqs. (stok_eig), (Curl)).
* zeta = xhat . Curl_n u = sum lambda_L^{1/2} alpha_{L,m} Y_{L,m}
  (Eq. (vort_app): Psi_N = -sum lambda^{-1/2} alpha Y, zeta = Delta Psi_N).
* Eq. (short_nonlin1): grad_u u = Grad(|u|^2/2) - u x Curl_n u, and
  -u x (zeta xhat) = zeta xhat x u.  The gradient is L^2-orthogonal to every
  Z_{L,m} (Eq. (div_thm)); with M >= 3N+2 (Eq. (M_choice)) Q_M integrates the
  remaining products exactly, so it drops out of the Galerkin system
  Eq. (app1_weak_form).
* Coriolis: C u = 2 Omega cos(theta) xhat x u (Eq. (C)), fused with the
  vorticity into one pointwise factor q = zeta + 2 Omega cos(theta).
* ( . , . )_M is the discrete inner product Eq. (disc_ip), with Q_M of
  Eq. (quadrule).
* fhat_{L,m} = (f, Z_{L,m})_M is passed in as packed coefficients.

In the orthonormal frame (e_theta, e_phi), xhat x e_theta = e_phi and
xhat x e_phi = -e_theta, and for Y = Pt_L^m(cos theta) e^{i m phi}:
  Grad Y = d_theta Y e_theta + (i m Y / sin theta) e_phi
  Curl Y = (i m Y / sin theta) e_theta - d_theta Y e_phi
so u_theta = sum alpha lambda^{-1/2} (i m / sin) Y and
u_phi = -sum alpha lambda^{-1/2} d_theta Y; W = q xhat x u has
W_theta = -q u_phi and W_phi = q u_theta.

Two independent evaluations:
  ``rhs_bruteforce``  every Z_{L,m} evaluated at every node (all signed m),
                      direct double sums (Eqs. (app_soln_rep), (disc_ip));
                      intended for N <= 31.
  ``rhs_separable``   per-order Legendre sums and a naive truncated DFT along
                      longitude (Sec. 4.2: the phi sums are Fourier sums); no
                      FFT and no blocking.
"""
import numpy as np

from . import layout
from .legendre import (dtheta_from_degree_shift, dtheta_from_order_ladder,
                       pt_bruteforce_signed, pt_table)
from .quadrature import Grid


class Problem:
    """Truncation N, quadrature parameter M (grid M/2 x M), nu, Omega."""

    def __init__(self, N, M, nu, Omega):
        self.N, self.M = int(N), int(M)
        self.nu, self.Omega = float(nu), float(Omega)
        self.grid = Grid(self.M)
        self.Ls, self.ms = layout.packed_degrees_orders(self.N)
        self.off = layout.order_offsets(self.N)
        self.lam = (self.Ls * (self.Ls + 1)).astype(np.float64)
        self._tables = None

    # ------------------------------------------------------------------
    # Legendre tables for the separable evaluation (built once, lazily)
    def tables(self):
        if self._tables is None:
            g = self.grid
            ext = pt_table(self.N + 1, g.x, g.sin)
            dth = dtheta_from_degree_shift(ext, self.N, g.sin)
            self._tables = ([t[: self.N - m + 1] for m, t in enumerate(ext[: self.N + 1])], dth)
        return self._tables

    def n(self):
        return layout.n_packed(self.N)


# ----------------------------------------------------------------------
# separable evaluation (per-order Legendre sums + naive DFT)

def _dft_matrix(M, orders, sign):
    """E[m, q] = exp(sign * i * m * phi_q), angles reduced exactly:
    m q mod M is an integer."""
    q = np.arange(M)
    red = np.mod(np.outer(np.asarray(orders, dtype=np.int64), q), M)
    ang = 2.0 * np.pi * red / M
    return np.cos(ang) + sign * 1j * np.sin(ang)


def spectral_fields(prob, alpha):
    """Per-order latitude profiles g_m(theta_p), m = 0..N, of zeta, u_theta,
    u_phi (complex, shape (N+1, nlat) each)."""
    P, D = prob.tables()
    g = prob.grid
    N = prob.N
    zeta = np.zeros((N + 1, g.nlat), dtype=np.complex128)
    uth = np.zeros_like(zeta)
    uph = np.zeros_like(zeta)
    for m in range(N + 1):
        a = alpha[prob.off[m]: prob.off[m + 1]]
        Ls = np.arange(max(m, 1), N + 1)
        lam = Ls * (Ls + 1.0)
        rows = Ls - m
        Pm, Dm = P[m][rows], D[m][rows]
        zeta[m] = (np.sqrt(lam) * a) @ Pm
        uth[m] = (1j * m / g.sin) * ((a / np.sqrt(lam)) @ Pm)
        uph[m] = -((a / np.sqrt(lam)) @ Dm)
    return zeta, uth, uph


def to_grid(prob, gm):
    """field(theta_p, phi_q) = sum_{m=-N}^{N} g_m(theta_p) e^{i m phi_q} with
    g_{-m} = conj(g_m) (real field).  Returns (real grid, max |imag|)."""
    N, M = prob.N, prob.M
    orders = np.arange(-N, N + 1)
    full = np.concatenate([np.conj(gm[:0:-1]), gm], axis=0)  # m = -N..N
    f = full.T @ _dft_matrix(M, orders, +1.0)
    return f.real, float(np.max(np.abs(f.imag))) if f.size else 0.0


def synthesize(prob, alpha):
    """Grid fields (zeta, u_theta, u_phi), each (nlat, M), real."""
    out = []
    for gm in spectral_fields(prob, alpha):
        f, _ = to_grid(prob, gm)
        out.append(f)
    return tuple(out)


def from_grid(prob, W):
    """Ghat_m(theta_p) = (2 pi / M) sum_q W(theta_p, phi_q) e^{-i m phi_q},
    m = 0..N; shape (N+1, nlat)."""
    E = _dft_matrix(prob.M, np.arange(prob.N + 1), -1.0)
    return (2.0 * np.pi / prob.M) * (E @ W.T)


def project(prob, W_theta, W_phi):
    """Packed (W, Z_{L,m})_M = Q_M(W . conj Z_{L,m}) (Eq. (disc_vec_orth_proj))
    with conj Z_{L,m} = lambda^{-1/2} [(-i m / sin) conj Y, -d_theta conj Y]."""
    P, D = prob.tables()
    g = prob.grid
    N = prob.N
    Gt = from_grid(prob, W_theta)
    Gp = from_grid(prob, W_phi)
    out = np.zeros(prob.n(), dtype=np.complex128)
    for m in range(N + 1):
        Ls = np.arange(max(m, 1), N + 1)
        lam = Ls * (Ls + 1.0)
        rows = Ls - m
        Pm, Dm = P[m][rows], D[m][rows]
        val = Pm @ (g.w * (-1j * m / g.sin) * Gt[m]) - Dm @ (g.w * Gp[m])
        out[prob.off[m]: prob.off[m + 1]] = val / np.sqrt(lam)
    return out


def project_scalar(prob, rho):
    """Packed (rho, Y_{L,m})_M = Q_M(rho conj Y_{L,m}) for a real grid scalar
    (Eq. (disc_ip))."""
    P, _ = prob.tables()
    g = prob.grid
    G = from_grid(prob, rho)
    out = np.zeros(prob.n(), dtype=np.complex128)
    for m in range(prob.N + 1):
        Ls = np.arange(max(m, 1), prob.N + 1)
        out[prob.off[m]: prob.off[m + 1]] = P[m][Ls - m] @ (g.w * G[m])
    return out


def pointwise_product(prob, zeta, uth, uph):
    """W = (zeta + 2 Omega cos theta) xhat x u on the grid (Eqs. (short_nonlin1), (C))."""
    q = zeta + 2.0 * prob.Omega * prob.grid.x[:, None]
    return -q * uph, q * uth


def nonlinear_separable(prob, alpha):
    """N_{L,m} = ((zeta + 2 Omega cos) xhat x u, Z_{L,m})_M."""
    zeta, uth, uph = synthesize(prob, alpha)
    Wt, Wp = pointwise_product(prob, zeta, uth, uph)
    return project(prob, Wt, Wp)


def rhs_separable(prob, alpha, forcing=None):
    """F = fhat - nu lambda alpha - N (Eqs. (ode), (app1_weak_form))."""
    alpha = np.asarray(alpha, dtype=np.complex128)
    F = -prob.nu * prob.lam * alpha - nonlinear_separable(prob, alpha)
    if forcing is not None:
        F = F + np.asarray(forcing, dtype=np.complex128)
    return F


# ----------------------------------------------------------------------
# brute-force evaluation (every basis field at every node)

def basis_bruteforce(prob):
    """For every (L, m), |m| <= L <= N: Y, Z_theta, Z_phi on the grid,
    complex arrays of shape (nlat, M); keyed by (L, m)."""
    g = prob.grid
    out = {}
    for L in range(1, prob.N + 1):
        lam = L * (L + 1.0)
        for m in range(-L, L + 1):
            e = np.exp(1j * m * g.phi)[None, :]
            pt = pt_bruteforce_signed(L, m, g.x, g.sin)[:, None]
            dpt = dtheta_from_order_ladder(L, m, g.x, g.sin)[:, None]
            Y = pt * e
            Zt = (1j * m / g.sin[:, None]) * Y / np.sqrt(lam)
            Zp = -dpt * e / np.sqrt(lam)
            out[(L, m)] = (Y, Zt, Zp)
    return out


def rhs_bruteforce(prob, alpha, forcing=None, basis=None, return_all=False):
    """F by direct sums over every mode and every node.  With
    ``return_all`` also returns N for negative orders and the grid fields."""
    g = prob.grid
    if basis is None:
        basis = basis_bruteforce(prob)
    full = layout.full_from_packed(np.asarray(alpha, dtype=np.complex128), prob.N)
    zeta = np.zeros((g.nlat, g.M), dtype=np.complex128)
    ut = np.zeros_like(zeta)
    up = np.zeros_like(zeta)
    for (L, m), (Y, Zt, Zp) in basis.items():
        a = full[(L, m)]
        zeta += np.sqrt(L * (L + 1.0)) * a * Y
        ut += a * Zt
        up += a * Zp
    imag = max(np.max(np.abs(zeta.imag)), np.max(np.abs(ut.imag)), np.max(np.abs(up.imag)))
    zeta, ut, up = zeta.real, ut.real, up.real
    q = zeta + 2.0 * prob.Omega * g.x[:, None]
    Wt, Wp = -q * up, q * ut
    wq = (2.0 * np.pi / g.M) * g.w[:, None]
    Nfull = {}
    for (L, m), (Y, Zt, Zp) in basis.items():
        Nfull[(L, m)] = np.sum(wq * (Wt * np.conj(Zt) + Wp * np.conj(Zp)))
    Nvec = np.array([Nfull[(int(L), int(m))] for L, m in zip(prob.Ls, prob.ms)])
    F = -prob.nu * prob.lam * np.asarray(alpha, dtype=np.complex128) - Nvec
    if forcing is not None:
        F = F + np.asarray(forcing, dtype=np.complex128)
    if return_all:
        return F, {"N": Nfull, "zeta": zeta, "u_theta": ut, "u_phi": up, "imag": imag}
    return F
