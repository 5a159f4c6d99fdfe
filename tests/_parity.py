"""Per-degree and per-order error of a computed RHS against the oracle's.

The global 2-norm of F hides errors in the high degrees whenever the input
spectrum decays, and the diagonal terms f - nu lambda alpha dilute it
further.  These helpers compare the nonlinear part
N = -(F - fhat + nu lambda alpha) degree by degree (all orders of one L) and
order by order (all degrees of one m):

  e_L = ||dN_L|| / max(||N_L||, floor * max_L' ||N_L'||)

and the same over orders.  With floor = 0 every degree counts at full weight;
a decaying spectrum needs a floor because rounding is uniform over the
coefficients while N_L falls by decades.  On a flat spectrum the low degrees
carry a small share of N (the advection moves little to the largest scales),
so there the floor is a degree's share of the norm, ||N|| sqrt(c_L / n) for
its c_L of the n coefficients: a rounding error spread evenly gives e_L near
the global relative error, and an error concentrated in one block does not.
"""
import numpy as np


def nonlinear_part(F, prob, alpha, forcing=None):
    N = -(np.asarray(F) + prob.nu * prob.lam * alpha)
    if forcing is not None:
        N = N + forcing
    return N


def _grouped(key, nbins, d2, r2, floor, kmin=0, share=False):
    de = np.sqrt(np.bincount(key, weights=d2, minlength=nbins))
    nr = np.sqrt(np.bincount(key, weights=r2, minlength=nbins))
    cnt = np.bincount(key, minlength=nbins)
    present = (cnt > 0) & (np.arange(nbins) >= kmin)
    den = np.maximum(nr, floor * nr.max())
    if share:
        den = np.maximum(den, np.sqrt(r2.sum() * cnt / key.size))
    e = np.where(present & (den > 0), de / np.where(den > 0, den, 1.0), 0.0)
    i = int(np.argmax(e))
    return float(e[i]), i


def degree_order_errors(got, ref, prob, alpha, forcing=None, floor=0.0, Lmin=1, share=False):
    """(max_L e_L, worst L, max_m e_m, worst m) of the nonlinear part;
    degrees below Lmin are left out of e_L; share: floor at each group's
    share of the norm (module docstring)."""
    Ng = nonlinear_part(got, prob, alpha, forcing)
    Nr = nonlinear_part(ref, prob, alpha, forcing)
    d2 = np.abs(Ng - Nr) ** 2
    r2 = np.abs(Nr) ** 2
    eL, Lw = _grouped(prob.Ls, prob.N + 1, d2, r2, floor, Lmin, share)
    em, mw = _grouped(prob.ms, prob.N + 1, d2, r2, floor, 0, share)
    return eL, Lw, em, mw


def degree1_defect(got, prob, alpha, forcing=None):
    """||N_1 - C_1|| / ||N||: the advection term has no degree-1 component
    (the angular momentum of the flow is conserved by it), so at L = 1 only
    the Coriolis diagonal 2 i Omega m / lambda alpha of Eq. (Coriolis_ZLm)
    remains in N (with the sign of N = -(F - fhat + nu lambda alpha))."""
    N = nonlinear_part(got, prob, alpha, forcing)
    cor = -2j * prob.Omega * prob.ms / prob.lam * alpha
    sel = prob.Ls == 1
    return float(np.linalg.norm((N - cor)[sel]) / np.linalg.norm(N))


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))
