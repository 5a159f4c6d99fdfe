"""Tangent-linear (forward-mode) model of F and of the frozen-controller NDF
step, and the final-time objective.  Oracle only.

Independent of any adjoint: gradients produced elsewhere are checked through
directional derivatives <grad J, v> = dJ(alpha_0 + eps v)/d eps computed here.

* F(alpha, nu) = fhat - nu lambda alpha - N(alpha) (Eq. (ode)) has
  dF = -nu lambda dalpha - dnu lambda alpha - dN, with
  dN = ( dzeta xhat x u + q xhat x du , Z_{L,m} )_M,  q = zeta + 2 Omega cos
  (derivative of the pointwise product of Eqs. (short_nonlin1), (C)).
* The NDF corrector c F(alpha^(0) + d) - psi - d = 0 (Eq. (ode_disc), written
  as in ``oracle.ndf``) gives
  (I - c J) dd = c (J dalpha^(0) + F_nu dnu) - dpsi,  J = dF/dalpha,
  solved by fixed-point iteration preconditioned with the diagonal
  iteration matrix I - c J_d.
* Objective (final time T):
  J = KE_band + sum_{all L, m} |alpha_{L,m}(T) - alpha*_{L,m}|^2,
  KE_band = 1/2 Q_M restricted to the nodes with colatitude in
  [theta_lo, theta_hi] of |u|^2 (a nodal mask; reading of "kinetic energy in
  a latitude band"); the second term is the L^2 misfit of the velocity by
  Parseval (the Z_{L,m} are orthonormal, Eq. (Fourier_coeff)).
"""
import numpy as np

from . import layout
from .ndf import NDF, rescale_matrix, _real
from .rhs import pointwise_product, project, synthesize


def rhs_tlm(prob, alpha, dalpha, dnu=0.0):
    """dF at (alpha, nu) in direction (dalpha, dnu)."""
    zeta, uth, uph = synthesize(prob, alpha)
    dz, dut, dup = synthesize(prob, dalpha)
    q = zeta + 2.0 * prob.Omega * prob.grid.x[:, None]
    # d[(zeta + f) xhat x u] = dzeta xhat x u + q xhat x du
    dWt = -dz * uph - q * dup
    dWp = dz * uth + q * dut
    dN = project(prob, dWt, dWp)
    return -prob.nu * prob.lam * dalpha - dnu * prob.lam * alpha - dN


def band_mask(prob, theta_lo, theta_hi):
    th = prob.grid.theta
    return ((th >= theta_lo) & (th <= theta_hi)).astype(np.float64)


def objective(prob, alpha, alpha_target, theta_lo, theta_hi):
    """J = KE_band + misfit (module docstring)."""
    _, uth, uph = synthesize(prob, alpha)
    g = prob.grid
    wq = (2.0 * np.pi / g.M) * (g.w * band_mask(prob, theta_lo, theta_hi))[:, None]
    ke = 0.5 * np.sum(wq * (uth ** 2 + uph ** 2))
    s = layout.multiplicity(prob.ms)
    mis = np.sum(s * np.abs(alpha - alpha_target) ** 2)
    return float(ke + mis)


def objective_tlm(prob, alpha, dalpha, alpha_target, theta_lo, theta_hi):
    _, uth, uph = synthesize(prob, alpha)
    _, dut, dup = synthesize(prob, dalpha)
    g = prob.grid
    wq = (2.0 * np.pi / g.M) * (g.w * band_mask(prob, theta_lo, theta_hi))[:, None]
    dke = np.sum(wq * (uth * dut + uph * dup))
    s = layout.multiplicity(prob.ms)
    dmis = 2.0 * np.sum(s * (np.conj(alpha - alpha_target) * dalpha).real)
    return float(dke + dmis)


class ReplayTLM:
    """Frozen-controller NDF trajectory with its tangent-linear model.

    ``ndf`` is an ``oracle.ndf.NDF`` freshly initialised at alpha_0 (with
    the initial difference D_0 = h0 F(t0, alpha_0)); the tangent state
    starts at (dalpha_0, dD_0 = h0 dF(alpha_0; dalpha_0, dnu)).
    """

    def __init__(self, prob, ndf: NDF, dalpha0, dnu=0.0, forcing=None):
        self.prob = prob
        self.ndf = ndf
        self.dnu = float(dnu)
        self.dy = np.array(dalpha0, dtype=np.complex128)
        self.dD = np.zeros_like(ndf.dif)
        self.dD[0] = ndf.h * rhs_tlm(prob, ndf.y, self.dy, self.dnu)

    def _jvp(self, alpha, v):
        return rhs_tlm(self.prob, alpha, v, 0.0)

    def step(self, h, k, tol=1e-15, maxit=200):
        nd = self.ndf
        c = nd.c
        # rescale (linear) -- must use the pre-step h of the forward state
        if h != nd.h_dif:
            self.dD[:k] = rescale_matrix(k, h / nd.h_dif).T @ self.dD[:k]
        nd.replay_step(h, k)
        ynew = nd.y
        dy0 = self.dy + self.dD[:k].sum(axis=0)
        dpsi = (np.array([c.g(j + 1) for j in range(k)]) @ self.dD[:k]) * c.iga(k)
        cc = h * c.iga(k)
        miter = 1.0 - cc * nd.jdiag
        fnu = -self.prob.lam * ynew
        base = cc * (self._jvp(ynew, dy0) + fnu * self.dnu) - dpsi
        dd = np.zeros_like(dy0)
        scale = max(np.max(np.abs(base)), 1e-300)
        for _ in range(maxit):
            r = base + cc * self._jvp(ynew, dd) - dd
            dd = dd + r / miter
            if np.max(np.abs(r)) <= tol * scale:
                break
        D = self.dD
        D[k + 1] = dd - D[k]
        D[k] = dd
        for j in range(k - 1, -1, -1):
            D[j] = D[j] + D[j + 1]
        self.dy = dy0 + dd
        return self.dy
