"""Seeded synthetic inputs for the rotating-sphere Navier-Stokes workloads.

This module only draws random numbers and arranges them in the packed
coefficient order; it holds none of the method's arithmetic.  Both the CUDA
path (through its tests and ``bench.py``) and the CPU oracle consume what it
returns, so neither side generates its own inputs.

Packed order of a coefficient vector for truncation N: m = 0..N, and for each
m the degrees L = max(m, 1)..N; complex128; alpha_{L,0} is real.

Spectra (stand-ins for the random Gevrey-decaying initial state of the
paper's Sec. 5 Example 2): alpha_{L,m} = sigma_L (g1 + i g2)/sqrt(2) for
m >= 1 and sigma_L g1 for m = 0, g ~ N(0, 1) from numpy's Philox generator.
"""
import math

import numpy as np


def packed_orders(N):
    """(L, m) integer arrays in packed order."""
    Ls, ms = [], []
    for m in range(N + 1):
        for L in range(max(m, 1), N + 1):
            Ls.append(L)
            ms.append(m)
    return np.array(Ls, dtype=np.int64), np.array(ms, dtype=np.int64)


def _draw(rng, N, sigma_of_L, mask=None):
    Ls, ms = packed_orders(N)
    g = rng.standard_normal((Ls.size, 2))
    sig = np.array([sigma_of_L(int(L)) for L in Ls], dtype=np.float64)
    a = np.where(ms == 0, sig * g[:, 0],
                 sig * (g[:, 0] + 1j * g[:, 1]) / math.sqrt(2.0))
    a = a.astype(np.complex128)
    if mask is not None:
        a = np.where(mask(Ls, ms), a, 0.0)
    return a


def gevrey(decay):
    """sigma_L = exp(-decay L) / (L (L + 1))."""
    return lambda L: math.exp(-decay * L) / (L * (L + 1.0))


def coefficients(N, seed, decay):
    """Random packed coefficients with sigma_L = exp(-decay L)/(L(L+1))."""
    rng = np.random.Generator(np.random.Philox(seed))
    return _draw(rng, N, gevrey(decay))


# --------------------------------------------------------------------------
# the five workloads (sizes, physical parameters, seeds)

CONFIGS = {
    # FP64, L = 31, 48 x 96, 100 adaptive steps, rtol 1e-8, steady forcing
    "L31": dict(L=31, nlat=48, nlon=96, nu=1e-2, Omega=1.0, seed=1, decay=0.3,
                forcing_Lmax=4, rtol=1e-8, steps=100),
    # FP64 on the GPU, L = 255, 384 x 768, 1000 RHS evaluations
    "L255": dict(L=255, nlat=384, nlon=768, nu=1e-4, Omega=1.0, seed=2, decay=0.05,
                 forcing_Lmax=0, rtol=1e-6, steps=0),
    # mixed precision, L = 511, 768 x 1536, 500 steps
    "L511": dict(L=511, nlat=768, nlon=1536, nu=5e-5, Omega=1.0, seed=3, decay=0.02,
                 forcing_Lmax=0, rtol=1e-6, steps=500),
    # adjoint, L = 255, 200 steps, checkpoints every 20
    "adjoint": dict(L=255, nlat=384, nlon=768, nu=1e-4, Omega=1.0, seed=5, decay=0.05,
                    target_seed=55, forcing_Lmax=0, rtol=1e-6, steps=200, checkpoint=20),
}


def workload(name):
    """Initial coefficients (and steady forcing, target) of a named workload."""
    c = dict(CONFIGS[name])
    rng = np.random.Generator(np.random.Philox(c["seed"]))
    N = c["L"]
    out = {"config": c, "alpha0": _draw(rng, N, gevrey(c["decay"]))}
    if c.get("forcing_Lmax", 0) > 0:
        nu, Lf = c["nu"], c["forcing_Lmax"]
        # steady forcing at L <= Lf, sigma^f_L = nu exp(-decay L), same stream
        out["forcing"] = _draw(rng, N, lambda L: nu * math.exp(-c["decay"] * L),
                               mask=lambda Ls, ms: Ls <= Lf)
    else:
        out["forcing"] = None
    if "target_seed" in c:
        out["target"] = coefficients(N, c["target_seed"], c["decay"])
    return out


def example2(N=100, seed=2020, nu=1e-4, Lmax=20):
    """Initial state of Sec. 5 Example 2: alpha_{L,m} = a_L exp(i phi_{L,m})
    for L <= Lmax and m >= 0 (phi_{L,0} = 0; reading: an independent phase
    per (L, m)), zero above Lmax; a_L = b_L / ||b||, b_L = 2 / (L + (nu L)^2.5).
    Negative orders follow from the packed symmetry."""
    rng = np.random.Generator(np.random.Philox(seed))
    Ls, ms = packed_orders(N)
    b = np.array([2.0 / (L + (nu * L) ** 2.5) for L in range(1, Lmax + 1)])
    a = b / np.linalg.norm(b)
    phi = rng.uniform(0.0, 2.0 * math.pi, size=Ls.size)
    phi[ms == 0] = 0.0
    amp = np.where(Ls <= Lmax, a[np.minimum(Ls, Lmax) - 1], 0.0)
    return (amp * np.exp(1j * phi)).astype(np.complex128)


def example2_forcing_30(t):
    """The only nonzero forcing coefficient of Example 2, fhat_{3,0}(t)."""
    return 1.0 if t <= 10.0 else math.cos(math.pi * t / 5.0) * math.exp(-(t - 10.0) / 5.0)


def ensemble(n_instances=256, degrees=(63, 127, 255), seed0=1000, decay=0.05,
             nu_range=(1e-5, 1e-3)):
    """Batched-ensemble members: per instance a truncation drawn uniformly
    from ``degrees`` (grid 3(L+1)/2 x 3(L+1)), nu log-uniform in
    ``nu_range`` and coefficients from seed ``seed0 + i``."""
    rng = np.random.Generator(np.random.Philox(seed0 - 1))
    Ls = rng.choice(np.array(degrees), size=n_instances)
    lo, hi = math.log10(nu_range[0]), math.log10(nu_range[1])
    nus = 10.0 ** rng.uniform(lo, hi, size=n_instances)
    members = []
    for i in range(n_instances):
        L = int(Ls[i])
        members.append(dict(L=L, nlat=3 * (L + 1) // 2, nlon=3 * (L + 1),
                            nu=float(nus[i]), Omega=1.0,
                            alpha0=coefficients(L, seed0 + i, decay)))
    return members


def random_packed(N, seed, scale=1.0):
    """Unit-variance random packed vector (directions, adjoint seeds)."""
    rng = np.random.Generator(np.random.Philox(seed))
    return _draw(rng, N, lambda L: scale)
