"""Plain, slow FP64 CPU oracle for the pseudospectral quadrature method.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import or call
this package: only ``tests/``, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` use it.  It shares no code with the CUDA path
(``paper_1009_3308_gb300``) and imports nothing from it.

What it computes (Ganesh, Le Gia & Sloan, "A pseudospectral quadrature method
for Navier-Stokes equations on rotating spheres"):

* ``quadrature``   Gauss-rectangle rule Q_M of Eq. (quadrule), Sec. 3.
* ``legendre``     orthonormal associated Legendre functions behind the
                   scalar harmonics Y_{L,m} of Eq. (sph_har), Sec. 2.
* ``layout``       packed coefficient order (m >= 0 only, Hermitian
                   symmetry of Eq. (app_soln_rep)).
* ``rhs``          F(t, alpha) of Eq. (ode): the Galerkin system
                   Eq. (app1_weak_form) with the nonlinear term rewritten by
                   Eq. (short_nonlin1) and the Coriolis operator of Eq. (C).
                   Two independent evaluations: ``rhs_bruteforce`` (direct
                   evaluation of every Z_{L,m} at every node) and
                   ``rhs_separable`` (per-order Legendre sums and a naive
                   truncated DFT, no FFT).
* ``tlm``          tangent-linear (forward-mode) derivative of F.
* ``ndf``          variable-order NDF integrator of Eq. (ode_disc), Sec. 4.2.

All floating point is IEEE binary64.  Every function names the passage of
the paper it follows.  Where the paper is silent or inconsistent the reading
taken is stated in the function's docstring.
"""
