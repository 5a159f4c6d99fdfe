"""Associated Legendre functions for the scalar harmonics of Eq. (sph_har).
Oracle only.

Convention (reading of Eq. (sph_har), Sec. 2): for m >= 0

    Y_{L,m}(theta, phi) = Pt_L^m(cos theta) e^{i m phi},
    Pt_L^m = [(2L+1)/(4 pi) (L-m)!/(L+m)!]^{1/2} P_L^m,

with the Condon-Shortley phase (-1)^m inside P_L^m, and for negative order
Y_{L,-m} = (-1)^m conj(Y_{L,m}), the relation printed under Eq. (sph_har).

Two independent evaluations are provided:

* ``pt_table``     the orthonormal three-term recurrence in L, carried with
                   an extended binary exponent so that sin(theta)^m never
                   underflows mid-recurrence (the paper stops at N = 100 and
                   is silent on this; values below the binary64 range come
                   out as 0 or subnormal, as ldexp rounds them);
* ``pt_bruteforce`` the unnormalised recurrence for P_L^m times the
                   factorial normalisation of Eq. (sph_har) (small L only).

theta-derivatives, also two ways:

* ``dtheta_from_degree_shift``: sin(theta) d/dtheta Pt_L^m
      = L eps_{L+1,m} Pt_{L+1}^m - (L+1) eps_{L,m} Pt_{L-1}^m,
  eps_{L,m} = sqrt((L^2 - m^2) / (4 L^2 - 1))   (textbook relation);
* ``dtheta_from_order_ladder``: d/dtheta Pt_L^m
      = 1/2 [ sqrt((L-m)(L+m+1)) Pt_L^{m+1} - sqrt((L+m)(L-m+1)) Pt_L^{m-1} ]
  from the angular-momentum ladder operators, with Pt_L^{-1} = -Pt_L^1.
"""
import math

import numpy as np


def eps(L, m):
    """eps_{L,m} = sqrt((L^2 - m^2) / (4 L^2 - 1)); zero when L <= |m|."""
    L = np.asarray(L, dtype=np.float64)
    m = np.asarray(m, dtype=np.float64)
    num = np.maximum(L * L - m * m, 0.0)
    return np.sqrt(num / (4.0 * L * L - 1.0))


_RESCALE = 2.0 ** 200


def pt_table(Lmax, x, s):
    """Orthonormal Pt_K^m(x) for 0 <= m <= K <= Lmax at nodes x (sin = s).

    Returns a list ``T`` with ``T[m]`` of shape (Lmax - m + 1, len(x)) and
    ``T[m][K - m] = Pt_K^m(x)``.

    Steps (orthonormal recurrences, in the order a textbook states them):
      Pt_0^0 = 1/sqrt(4 pi)
      Pt_m^m = -sqrt((2m+1)/(2m)) sin(theta) Pt_{m-1}^{m-1}
      Pt_{m+1}^m = sqrt(2m+3) x Pt_m^m
      eps_{K,m} Pt_K^m = x Pt_{K-1}^m - eps_{K-1,m} Pt_{K-2}^m
    Each value is a mantissa times 2**e with an integer e shared by the two
    values the recurrence carries.
    """
    x = np.asarray(x, dtype=np.float64)
    s = np.asarray(s, dtype=np.float64)
    nx = x.size
    # diagonal Pt_m^m as (mantissa, exponent)
    diag_mant = np.empty((Lmax + 1, nx))
    diag_exp = np.zeros((Lmax + 1, nx), dtype=np.int64)
    mant = np.full(nx, 1.0 / math.sqrt(4.0 * math.pi))
    ex = np.zeros(nx, dtype=np.int64)
    diag_mant[0] = mant
    for m in range(1, Lmax + 1):
        mant = -math.sqrt((2.0 * m + 1.0) / (2.0 * m)) * s * mant
        fr, e2 = np.frexp(mant)
        mant, ex = fr, ex + e2
        diag_mant[m] = mant
        diag_exp[m] = ex
    table = []
    for m in range(Lmax + 1):
        out = np.empty((Lmax - m + 1, nx))
        p2 = np.zeros(nx)               # Pt_{K-2}^m mantissa
        p1 = diag_mant[m].copy()        # Pt_{K-1}^m mantissa
        e = diag_exp[m].copy()          # shared exponent
        out[0] = np.ldexp(p1, e)
        for K in range(m + 1, Lmax + 1):
            if K == m + 1:
                p0 = math.sqrt(2.0 * m + 3.0) * x * p1
            else:
                p0 = (x * p1 - float(eps(K - 1, m)) * p2) / float(eps(K, m))
            p2, p1 = p1, p0
            big = np.abs(p1) > _RESCALE
            if np.any(big):
                p1 = np.where(big, p1 / _RESCALE, p1)
                p2 = np.where(big, p2 / _RESCALE, p2)
                e = e + np.where(big, 200, 0)
            out[K - m] = np.ldexp(p1, e)
        table.append(out)
    return table


def dtheta_from_degree_shift(table_ext, Lmax, s):
    """d/dtheta Pt_L^m for 0 <= m <= L <= Lmax from a table that reaches
    degree Lmax + 1 (``pt_table(Lmax + 1, ...)``), via the degree-shift
    relation in the module docstring.  Returns the same list layout."""
    out = []
    for m in range(Lmax + 1):
        Tm = table_ext[m]
        d = np.empty((Lmax - m + 1, Tm.shape[1]))
        for L in range(m, Lmax + 1):
            up = Tm[L + 1 - m]
            down = Tm[L - 1 - m] if L - 1 >= m else 0.0
            d[L - m] = (L * float(eps(L + 1, m)) * up
                        - (L + 1) * float(eps(L, m)) * down) / s
        out.append(d)
    return out


def pt_bruteforce(L, m, x, s):
    """Pt_L^m(x), 0 <= m <= L, from the unnormalised recurrence for P_L^m
    (with Condon-Shortley phase) and the factorial normalisation of
    Eq. (sph_har).  Plain FP64; intended for L <= 40."""
    x = np.asarray(x, dtype=np.float64)
    s = np.asarray(s, dtype=np.float64)
    # P_m^m = (-1)^m (2m-1)!! sin^m
    dfact = 1.0
    for k in range(1, 2 * m, 2):
        dfact *= k
    pmm = (-1.0) ** m * dfact * s ** m
    if L == m:
        p = pmm
    else:
        p_prev, p = pmm, x * (2 * m + 1) * pmm
        for K in range(m + 2, L + 1):
            # (K - m) P_K^m = (2K - 1) x P_{K-1}^m - (K + m - 1) P_{K-2}^m
            p_prev, p = p, ((2 * K - 1) * x * p - (K + m - 1) * p_prev) / (K - m)
    norm = math.sqrt((2 * L + 1) / (4 * math.pi)
                     * math.factorial(L - m) / math.factorial(L + m))
    return norm * p


def pt_bruteforce_signed(L, m, x, s):
    """Pt_L^m for signed m, with Pt_L^{-m} = (-1)^m Pt_L^m (theta part of
    Y_{L,-m} = (-1)^m conj Y_{L,m})."""
    if abs(m) > L:
        return np.zeros_like(np.asarray(x, dtype=np.float64))
    if m >= 0:
        return pt_bruteforce(L, m, x, s)
    return (-1.0) ** (-m) * pt_bruteforce(L, -m, x, s)


def dtheta_from_order_ladder(L, m, x, s):
    """d/dtheta Pt_L^m (signed m allowed) from the ladder-operator relation
    in the module docstring, built on ``pt_bruteforce``."""
    up = pt_bruteforce_signed(L, m + 1, x, s)
    down = pt_bruteforce_signed(L, m - 1, x, s)
    return 0.5 * (math.sqrt(max((L - m) * (L + m + 1), 0)) * up
                  - math.sqrt(max((L + m) * (L - m + 1), 0)) * down)
