"""Gauss-rectangle quadrature Q_M (Sec. 3, Eq. (quadrule)).  Oracle only.

Q_M(psi) = (2 pi / M) * sum_{q} sum_{p=1}^{M/2} w_p psi(theta_p, phi_q)

with cos(theta_p), w_p the M/2-point Gauss-Legendre nodes and weights on
[-1, 1] and phi_q = 2 q pi / M.  The paper numbers q = 1..M; q = 0..M-1 is the
same set of angles modulo 2 pi.

Pinned in tests against: exactness on x^k for k <= M-1, sum of weights = 2,
numpy's ``leggauss`` (test-only library routine).
"""
import numpy as np


def _legendre_near_north(n, theta):
    """(P_n, D_n = P_n - P_{n-1}) at x = cos(theta), evaluated through
    y = 1 - x = 2 sin^2(theta/2) so that no 1 - x cancellation occurs:
    Bonnet's recurrence (k+1) P_{k+1} = (2k+1) x P_k - k P_{k-1} rewritten as
    (k+1) D_{k+1} = k D_k - (2k+1) y P_k,  P_{k+1} = P_k + D_{k+1}."""
    y = 2.0 * np.sin(0.5 * theta) ** 2
    p = 1.0 - y            # P_1
    d = -y                 # P_1 - P_0
    for k in range(1, n):
        d = (k * d - (2 * k + 1) * y * p) / (k + 1)
        p = p + d
    return p, d, y


def gauss_legendre(n):
    """n-point Gauss-Legendre rule on [-1, 1], nodes ordered north to south.

    Newton's method in the colatitude theta on f(theta) = P_n(cos theta) for
    the northern nodes, with
      d/dtheta P_n(cos theta) = n (x P_n - P_{n-1}) / sin(theta)
                              = n (D_n - y P_n) / sin(theta)
    (from (1 - x^2) P_n' = n (P_{n-1} - x P_n)); the southern nodes are the
    mirror images theta -> pi - theta.  Weights
      w = 2 / ((1 - x^2) P_n'(x)^2) = 2 sin^2(theta) / (n (D_n - y P_n))^2.
    Returns (theta, x, sin_theta, w), x descending.
    """
    nh = (n + 1) // 2
    i = np.arange(1, nh + 1, dtype=np.float64)
    theta = np.pi * (i - 0.25) / (n + 0.5)  # textbook starting guess
    if n % 2:
        theta[-1] = 0.5 * np.pi             # the equator is a node for odd n
    for _ in range(100):
        p, d, y = _legendre_near_north(n, theta)
        step = p * np.sin(theta) / (n * (d - y * p))
        if n % 2:
            step[-1] = 0.0
        theta = theta - step
        if np.max(np.abs(step)) <= 1e-16 * np.max(theta):
            break
    p, d, y = _legendre_near_north(n, theta)
    s = np.sin(theta)
    w = 2.0 * s * s / (n * (d - y * p)) ** 2
    m = n // 2
    theta_all = np.concatenate([theta, np.pi - theta[:m][::-1]])
    w_all = np.concatenate([w, w[:m][::-1]])
    x_all = np.concatenate([np.cos(theta), -np.cos(theta[:m][::-1])])
    s_all = np.concatenate([s, s[:m][::-1]])
    if n % 2:
        x_all[nh - 1] = 0.0
    return theta_all, x_all, s_all, w_all


class Grid:
    """Nodes of Q_M for an even M: nlat = M/2 Gauss latitudes x M longitudes."""

    def __init__(self, M):
        if M < 2 or M % 2:
            raise ValueError("M must be an even integer >= 2")
        self.M = M
        self.nlat = M // 2
        self.theta, self.x, self.sin, self.w = gauss_legendre(self.nlat)
        self.phi = 2.0 * np.pi * np.arange(M) / M

    def integrate(self, values):
        """Q_M applied to grid values shaped (nlat, M) (Eq. (quadrule))."""
        return (2.0 * np.pi / self.M) * np.einsum("p,pq->", self.w, values)
