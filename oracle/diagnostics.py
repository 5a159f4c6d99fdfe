"""Diagnostics of Sec. 6.2 (energy spectrum of the solution).  Oracle only.

* ``energy_spectrum``: E(L) = sum_{|m| <= L} |beta_{L,m}|^2 of a field
  u = sum beta_{L,m} Z_{L,m}, Eq. (energy).  Packed coefficients hold m >= 0;
  |alpha_{L,-m}| = |alpha_{L,m}| under the symmetry of Eq. (app_soln_rep), so
  an order m > 0 counts twice.
* ``truncate``: P_{N1} u, the modes of degree <= N1 (Eq. (eq: cut_app_soln)).
* ``resize``: the same field in the packed layout of another truncation
  (coefficients above the new degree dropped, new ones zero).
* ``inertial_manifold``: the approximate inertial manifold of Eq. (eq:p-p),
  Phi(u1) = (nu A + C)^{-1} (P_{N2} - P_{N1}) [f - B(u1, u1)] for u1 = P_{N1} u1
  and N2 > N1, in coefficients of degree N2.  A acts on Z_{L,m} as lambda_L
  (Eq. (stok_eig)) and C as -2 i Omega m / lambda_L (Eq. (Coriolis_ZLm)).
  Modes above N1 of u1 are zero, so C u1 vanishes there and
  f - B(u1, u1) = fhat - N(u1) = F(u1) + nu lambda u1 = F(u1) on the band
  N1 < L <= N2, with F the RHS of Eq. (ode) at truncation N2.
"""
import numpy as np

from . import layout
from .rhs import rhs_separable


def energy_spectrum(N, alpha):
    """E(L) for L = 0..N (E(0) = 0), Eq. (energy)."""
    Ls, ms = layout.packed_degrees_orders(N)
    a = np.asarray(alpha, dtype=np.complex128)
    E = np.zeros(N + 1)
    np.add.at(E, Ls, layout.multiplicity(ms) * np.abs(a) ** 2)
    return E


def truncate(N, alpha, N1):
    """P_{N1} alpha in the degree-N layout."""
    Ls, _ = layout.packed_degrees_orders(N)
    return np.where(Ls <= N1, np.asarray(alpha, dtype=np.complex128), 0.0)


def resize(N_in, alpha, N_out):
    """alpha (degree N_in) in the packed layout of degree N_out."""
    src = {(int(L), int(m)): a for a, L, m in zip(alpha, *layout.packed_degrees_orders(N_in))}
    Ls, ms = layout.packed_degrees_orders(N_out)
    return np.array([src.get((int(L), int(m)), 0.0) for L, m in zip(Ls, ms)], dtype=np.complex128)


def inertial_manifold(prob, N1, alpha, forcing=None):
    """Phi of Eq. (eq:p-p) with N2 = prob.N: coefficients of degree N2, nonzero
    only for N1 < L <= N2.  alpha: degree-N2 packed; its modes above N1 are
    dropped first (u1 = P_{N1} u)."""
    u1 = truncate(prob.N, alpha, N1)
    F = rhs_separable(prob, u1, forcing)
    band = prob.Ls > N1
    res = prob.nu * prob.lam - 2j * prob.Omega * prob.ms / prob.lam   # (nu A + C) on Z_{L,m}
    out = np.zeros_like(F)
    out[band] = F[band] / res[band]
    return out
