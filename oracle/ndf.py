"""Variable-order, variable-step NDF integrator (Sec. 4.2, Eq. (ode_disc)).
Oracle only.

The paper integrates d alpha/dt = F(t, alpha) with the numerical
differentiation formulas NDF1..NDF5,

  sum_{j=1}^{p} (1/j) nabla^j alpha_{n+1}
        = h F(t_{n+1}, alpha_{n+1}) + kappa_p gamma_p nabla^{p+1} alpha_{n+1},
  gamma_p = sum_{j=1}^{p} 1/j,
  kappa = (-0.1850, -1/9, -0.0823, -0.0415, 0)   (kappa = 0: BDF),

"following details in" the MATLAB ODE suite (Shampine & Reichelt, 1997).
The paper gives no more; the reading taken here (the published description
of that suite's quasi-constant-step NDF code) is:

* backward differences D_j = nabla^{j+1} alpha_n are kept; predictor
  alpha^(0) = alpha_n + sum_{j<k} D_j;
* the corrector is written in terms of d = alpha_{n+1} - alpha^(0):
      c F(t_{n+1}, alpha^(0) + d) - psi - d = 0,
      c = h / ((1 - kappa_k) gamma_k),
      psi = sum_{j<k} gamma_{j+1} D_j / ((1 - kappa_k) gamma_k);
* simplified Newton with the diagonal linear part of F as iteration matrix,
      J_d = diag(-nu lambda_L + 2 i Omega m / lambda_L)
  (Eq. (Coriolis_ZLm) and the Stokes eigenvalues), at most 4 iterations,
  with the suite's rate test;
* local error estimate err = (kappa_k gamma_k + 1/(k+1)) ||d / wt||_inf with
  wt = max(|alpha_n|, |alpha_{n+1}|, atol/rtol) per real component;
* step rejection, order and step-size selection from the error estimates of
  orders k-1, k, k+1 with the suite's safety factors 1.2, 1.3, 1.4, and
  rescaling of the differences on a step-size change with the published
  interpolation matrices R(rho) U.

All arithmetic is FP64.  The state vector is the packed complex coefficient
vector; norms and weights act on its real and imaginary parts separately
(the N^2 + 2N real unknowns of Eq. (ode)).
"""
import math

import numpy as np

KAPPA_NDF = (-0.1850, -1.0 / 9.0, -0.0823, -0.0415, 0.0)
MAXK = 5


class Constants:
    def __init__(self, bdf=False):
        k = np.arange(1, MAXK + 1, dtype=np.float64)
        self.kappa = np.zeros(MAXK) if bdf else np.array(KAPPA_NDF)
        self.gamma = np.cumsum(1.0 / k)                  # gamma_k, k = 1..5
        self.inv_ga = 1.0 / (self.gamma * (1.0 - self.kappa))
        self.erconst = self.kappa * self.gamma + 1.0 / (k + 1.0)

    # 1-based accessors
    def g(self, k):
        return self.gamma[k - 1]

    def iga(self, k):
        return self.inv_ga[k - 1]

    def ec(self, k):
        return self.erconst[k - 1]


def rescale_matrix(k, rho):
    """(R(rho) U)[:k, :k]:  R_ij = prod_{l=1}^{i} (l - 1 - j rho) / l and
    U = R(1); right-multiplying the first k backward differences by it
    re-expresses them on the step h_new = rho h_old."""
    i = np.arange(1, k + 1, dtype=np.float64)[:, None]
    j = np.arange(1, k + 1, dtype=np.float64)[None, :]
    R = np.cumprod((i - 1.0 - j * rho) / i, axis=0)
    U = np.cumprod((i - 1.0 - j) / i, axis=0)
    return R @ U


def _real(v):
    return np.asarray(v).view(np.float64)


def wnorm(v, wt):
    """max-norm of v / wt over real components (v complex, wt real per
    component)."""
    return float(np.max(np.abs(_real(v)) / wt)) if v.size else 0.0


class NDF:
    """Adaptive NDF integrator state for d alpha/dt = F(t, alpha).

    rhs(t, alpha) -> F; jdiag: complex diagonal of the linear part of F.
    """

    def __init__(self, rhs, jdiag, t0, alpha0, rtol, atol, h0=None, h_max=1.0,
                 bdf=False, maxit=4, t_end=math.inf):
        self.rhs = rhs
        self.jdiag = np.asarray(jdiag, dtype=np.complex128)
        self.c = Constants(bdf)
        self.rtol, self.atol = float(rtol), float(atol)
        self.threshold = self.atol / self.rtol
        self.maxit = maxit
        self.h_max = h_max
        self.t_end = t_end
        self.t = float(t0)
        self.y = np.array(alpha0, dtype=np.complex128)
        n = self.y.size
        self.dif = np.zeros((MAXK + 2, n), dtype=np.complex128)
        f0 = rhs(self.t, self.y)
        self.nfev = 1
        if h0 is None or h0 <= 0:
            wt = np.maximum(np.abs(_real(self.y)), self.threshold)
            rh = 1.25 * float(np.max(np.abs(_real(f0)) / wt)) / math.sqrt(self.rtol)
            h0 = min(h_max, 1.0 / rh) if rh > 0 else h_max
        self.h = float(h0)
        self.k = 1
        self.dif[0] = self.h * f0
        self.h_dif = self.h        # step size the differences are expressed in
        self.nconhk = 0
        self.rate, self.havrate = 0.0, False
        self._miter_hk = None
        self.hmin_factor = 16.0 * np.finfo(np.float64).eps
        self.nsteps = 0
        self.nfailed = 0

    # --------------------------------------------------------------
    def _rescale_to(self, h):
        if h != self.h_dif:
            k = self.k
            self.dif[:k] = rescale_matrix(k, h / self.h_dif).T @ self.dif[:k]
            self.h_dif = h
            self.nconhk = 0

    def _corrector(self, h, k, tight=False, maxit=None):
        """Predictor and simplified-Newton corrector.  Returns
        (converged, y_new, d, n_iterations)."""
        c = self.c
        D = self.dif
        if (h, k) != self._miter_hk:
            # a new iteration matrix: forget the observed convergence rate
            self.havrate = False
            self._miter_hk = (h, k)
        y0 = self.y + D[:k].sum(axis=0)
        psi = (np.array([c.g(j + 1) for j in range(k)]) @ D[:k]) * c.iga(k)
        hinv = h * c.iga(k)
        miter = 1.0 - hinv * self.jdiag
        tnew = self.t + h
        d = np.zeros_like(self.y)
        ynew = y0.copy()
        minnrm = 100.0 * np.finfo(np.float64).eps * wnorm(
            self.y, np.maximum(np.abs(_real(self.y)), self.threshold))
        oldnrm = 0.0
        maxit = self.maxit if maxit is None else maxit
        for it in range(maxit):
            r = hinv * self.rhs(tnew, ynew) - (psi + d)
            self.nfev += 1
            dl = r / miter
            wt = np.maximum(np.maximum(np.abs(_real(self.y)), np.abs(_real(ynew))),
                            self.threshold)
            newnrm = wnorm(dl, wt)
            d = d + dl
            ynew = y0 + d
            if tight:
                if newnrm <= max(minnrm, 1e-15):
                    return True, ynew, d, it + 1
                continue
            if newnrm <= minnrm:
                return True, ynew, d, it + 1
            if it == 0:
                if self.havrate:
                    errit = newnrm * self.rate / (1.0 - self.rate)
                    if errit <= 0.05 * self.rtol:
                        return True, ynew, d, it + 1
                else:
                    self.rate = 0.0
            elif newnrm > 0.9 * oldnrm:
                return False, ynew, d, it + 1
            else:
                self.rate = max(0.9 * self.rate, newnrm / oldnrm)
                self.havrate = True
                errit = newnrm * self.rate / (1.0 - self.rate)
                if errit <= 0.5 * self.rtol:
                    return True, ynew, d, it + 1
                if it == maxit - 1:
                    return False, ynew, d, it + 1
                if 0.5 * self.rtol < errit * self.rate ** (maxit - 1 - it):
                    return False, ynew, d, it + 1
            oldnrm = newnrm
        return tight, ynew, d, maxit

    def _accept(self, k, h, ynew, d):
        D = self.dif
        D[k + 1] = d - D[k]
        D[k] = d
        for j in range(k - 1, -1, -1):
            D[j] = D[j] + D[j + 1]
        self.t = self.t + h
        self.y = ynew
        self.nsteps += 1

    # --------------------------------------------------------------
    def step(self):
        """One accepted step (with as many rejected attempts as needed).
        Returns a dict with t, h, order, newton iterations, err, rejections."""
        c = self.c
        nofailed = True
        rejections = 0
        newton_total = 0
        while True:
            hmin = self.hmin_factor * abs(self.t)
            h = min(self.h_max, max(hmin, self.h))
            if 1.1 * h >= self.t_end - self.t:
                h = self.t_end - self.t
            self.h = h
            self._rescale_to(h)
            k = self.k
            ok, ynew, d, its = self._corrector(h, k)
            newton_total += its
            if not ok:
                # the iteration matrix is exact for the linear part; shrink h
                self.nfailed += 1
                rejections += 1
                if h <= hmin:
                    raise RuntimeError("step size below minimum")
                self.h = max(hmin, 0.3 * h)
                continue
            wt = np.maximum(np.maximum(np.abs(_real(self.y)), np.abs(_real(ynew))),
                            self.threshold)
            err = wnorm(d, wt) * c.ec(k)
            if err > self.rtol:
                self.nfailed += 1
                rejections += 1
                if h <= hmin:
                    raise RuntimeError("step size below minimum")
                if nofailed:
                    nofailed = False
                    hopt = h * max(0.1, 0.833 * (self.rtol / err) ** (1.0 / (k + 1)))
                    if k > 1:
                        errkm1 = wnorm(self.dif[k - 1] + d, wt) * c.ec(k - 1)
                        hkm1 = h * max(0.1, 0.769 * (self.rtol / errkm1) ** (1.0 / k))
                        if hkm1 > hopt:
                            hopt = min(h, hkm1)
                            self.k = k - 1
                    self.h = max(hmin, hopt)
                else:
                    self.h = max(hmin, 0.5 * h)
                continue
            # accepted
            self._accept(k, h, ynew, d)
            info = {"t": self.t, "h": h, "order": k, "newton": newton_total,
                    "err": err, "rejections": rejections}
            self.nconhk = min(self.nconhk + 1, MAXK + 2)
            if self.nconhk >= k + 2:
                temp = 1.2 * (err / self.rtol) ** (1.0 / (k + 1))
                hopt = h / temp if temp > 0.1 else 10.0 * h
                kopt = k
                if k > 1:
                    errkm1 = wnorm(self.dif[k - 1], wt) * c.ec(k - 1)
                    temp = 1.3 * (errkm1 / self.rtol) ** (1.0 / k)
                    hkm1 = h / temp if temp > 0.1 else 10.0 * h
                    if hkm1 > hopt:
                        hopt, kopt = hkm1, k - 1
                if k < MAXK:
                    errkp1 = wnorm(self.dif[k + 1], wt) * c.ec(k + 1)
                    temp = 1.4 * (errkp1 / self.rtol) ** (1.0 / (k + 2))
                    hkp1 = h / temp if temp > 0.1 else 10.0 * h
                    if hkp1 > hopt:
                        hopt, kopt = hkp1, k + 1
                if hopt > h:
                    self.h = hopt
                    if kopt != k:
                        self.k = kopt
                        self.nconhk = 0
            return info

    # --------------------------------------------------------------
    def replay_step(self, h, k, maxit=50):
        """One step with the step size and order fixed by the caller (frozen
        controller), the corrector iterated to convergence.  The map
        (alpha_n, D) -> (alpha_{n+1}, D') this applies is the one the
        tangent-linear model differentiates."""
        self.k = k
        self._rescale_to(h)
        ok, ynew, d, its = self._corrector(h, k, tight=True, maxit=maxit)
        self._accept(k, h, ynew, d)
        return its
