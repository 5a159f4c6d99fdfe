"""Diagnostics of Sec. 6.2 on the GPU against the oracle: energy spectrum
(Eq. (energy)), truncation / resizing, and the approximate inertial manifold
(Eq. (eq:p-p)) at the paper's N1 = 3N/4, N2 = 2 N1 proportions."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle.diagnostics as D
from oracle.rhs import Problem
from seeded_inputs import coefficients

pytestmark = pytest.mark.gpu


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.complex128)).cuda()


@pytest.mark.parametrize("L,nlon", [(31, 96), (100, 324), (511, 1536)])
def test_energy_spectrum(L, nlon):
    from paper_1009_3308_gb300 import Plan
    a = coefficients(L, 600 + L, 0.02)
    plan = Plan(L, nlon // 2, nlon, 1e-4, 1.0)
    got = plan.energy_spectrum(_dev(a)).cpu().numpy()
    ref = D.energy_spectrum(L, a)
    np.testing.assert_allclose(got, ref, rtol=1e-13, atol=0)
    # deterministic
    np.testing.assert_array_equal(got, plan.energy_spectrum(_dev(a)).cpu().numpy())


def test_resize_and_truncate():
    from paper_1009_3308_gb300 import Plan
    a = coefficients(75, 7, 0.05)
    p150 = Plan(150, 243, 486, 1e-4, 1.0)
    p75 = Plan(75, 128, 256, 1e-4, 1.0)
    up = p150.resize(_dev(a), 75).cpu().numpy()
    np.testing.assert_array_equal(up, D.resize(75, a, 150))
    back = p75.resize(torch.from_numpy(up).cuda(), 150).cpu().numpy()
    np.testing.assert_array_equal(back, a)
    cut = p75.resize(_dev(a), 75, L_max=40).cpu().numpy()
    np.testing.assert_array_equal(cut, D.truncate(75, a, 40))


@pytest.mark.parametrize("N1,N2,nlon,prec,tol", [(24, 48, 162, "fp64", 1e-12), (75, 150, 486, "fp64", 1e-12),
                                                 (75, 150, 486, "fp32", 1e-5)])
def test_inertial_manifold(N1, N2, nlon, prec, tol):
    """Phi(P_{N1} u) at N2 = 2 N1 (the paper's choice) with steady forcing."""
    from paper_1009_3308_gb300 import Plan
    prob = Problem(N2, nlon, 1e-4, 1.0)
    a = D.resize(N1, coefficients(N1, 900 + N1, 0.05) * 3.0, N2)
    a = a + D.resize(N2, coefficients(N2, 901, 0.05), N2) * (prob.Ls > N1)   # modes above N1 are dropped
    f = coefficients(N2, 902, 0.3)
    ref = D.inertial_manifold(prob, N1, a, f)
    plan = Plan(N2, nlon // 2, nlon, 1e-4, 1.0, precision=prec)
    got = plan.inertial_manifold(N1, _dev(a), _dev(f)).cpu().numpy()
    # Phi (nu A + C) is the band part of F(u1), whose entries are small
    # against F's low modes: the error is stated relative to the whole F,
    # the quantity the RHS parity bound is about
    from oracle.rhs import rhs_separable
    F = rhs_separable(prob, D.truncate(N2, a, N1), f)
    res = prob.nu * prob.lam - 2j * prob.Omega * prob.ms / prob.lam
    err = np.linalg.norm((got - ref) * res) / np.linalg.norm(F)
    rel = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    print(f"N1={N1} N2={N2} {prec}: band RHS err vs |F| {err:.2e}, Phi rel err {rel:.2e}")
    assert err <= tol, err
    assert np.all(got[prob.Ls <= N1] == 0)


def test_inertial_manifold_arguments():
    from paper_1009_3308_gb300 import Plan, SphnseError
    plan = Plan(31, 48, 96, 1e-3, 1.0)
    a = _dev(coefficients(31, 1, 0.1))
    for n1 in (0, 31, 40):
        with pytest.raises(SphnseError):
            plan.inertial_manifold(n1, a)
