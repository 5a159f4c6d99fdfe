"""Packed coefficient order for alpha_{L,m}.  Oracle only.

The unknowns of Eq. (app_soln_rep) are alpha_{L,m}, L = 1..N, |m| <= L.
The field is real, so negative orders follow from the non-negative ones:
alpha_{L,-m} = (-1)^m conj(alpha_{L,m}) (reading of the symmetry printed with
Eq. (app_soln_rep), made consistent with conj Y_{L,m} = (-1)^m Y_{L,-m} of
Eq. (sph_har)), and alpha_{L,0} is real.

Packed order: m-major, m = 0..N, then L = max(m,1)..N; complex128.
n_c = (N+1)(N+2)/2 - 1 entries.
"""
import numpy as np


def packed_degrees_orders(N):
    """Arrays (L, m) of the packed entries, in packed order."""
    Ls, ms = [], []
    for m in range(N + 1):
        for L in range(max(m, 1), N + 1):
            Ls.append(L)
            ms.append(m)
    return np.array(Ls, dtype=np.int64), np.array(ms, dtype=np.int64)


def n_packed(N):
    return (N + 1) * (N + 2) // 2 - 1


def order_offsets(N):
    """off[m] = packed index of (L = max(m,1), m)."""
    off = np.zeros(N + 2, dtype=np.int64)
    for m in range(N + 1):
        off[m + 1] = off[m] + (N - max(m, 1) + 1)
    return off


def multiplicity(ms):
    """s_m = 1 for m = 0 and 2 for m > 0: how many (L, +-m) entries one
    packed coefficient stands for in a sum over all orders."""
    return np.where(np.asarray(ms) == 0, 1.0, 2.0)


def full_from_packed(alpha, N):
    """Dict (L, m) -> alpha_{L,m} for all |m| <= L using the symmetry above."""
    Ls, ms = packed_degrees_orders(N)
    out = {}
    for a, L, m in zip(alpha, Ls, ms):
        out[(int(L), int(m))] = complex(a)
        if m > 0:
            out[(int(L), -int(m))] = (-1.0) ** int(m) * np.conj(a)
    return out
