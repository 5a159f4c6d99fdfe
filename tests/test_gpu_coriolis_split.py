"""Split Coriolis variant: with SPHNSE_KEY_CORIOLIS_SPLIT the Coriolis term
is applied as its diagonal (C Z_{L,m}, Z_{L,m}) = -2 i Omega m / lambda_L
(Sec. 3, Eq. (Coriolis_ZLm)) and 2 Omega cos(theta) leaves the grid
product.  F must not change beyond rounding: FP64 against the oracle at
1e-12, the mixed paths against their unsplit form at their own error level."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle.rhs import Problem, rhs_separable
from seeded_inputs import coefficients, workload

pytestmark = pytest.mark.gpu


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.complex128)).cuda()


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("L,nlon,Om", [(31, 96, 1.0), (63, 192, 7.0), (127, 384, 1.0)])
def test_split_fp64_matches_oracle(L, nlon, Om):
    from paper_1009_3308_gb300 import Plan
    prob = Problem(L, nlon, 1e-3, Om)
    a = coefficients(L, 700 + L, 0.1) * 2.0
    f = coefficients(L, 800 + L, 0.3)
    ref = rhs_separable(prob, a, f)
    plan = Plan(L, nlon // 2, nlon, 1e-3, Om)
    plan.set("CORIOLIS_SPLIT", 1)
    assert plan.get("CORIOLIS_SPLIT") == 1
    got = plan.rhs(_dev(a), forcing=_dev(f)).cpu().numpy()
    err = _rel(got, ref)
    print(f"L={L} Omega={Om} split fp64 vs oracle {err:.2e}")
    assert err <= 1e-12, err


@pytest.mark.parametrize("prec,tol", [("fp32", 1e-6), ("bf16x3", 3e-5)])
def test_split_mixed_matches_unsplit(prec, tol):
    """L = 511 workload: split vs unsplit in the same precision, and split
    against the FP64 path."""
    from paper_1009_3308_gb300 import Plan
    w = workload("L511")
    c = w["config"]
    a = _dev(w["alpha0"])
    ref = Plan(c["L"], c["nlat"], c["nlon"], c["nu"], c["Omega"]).rhs(a).cpu().numpy()
    plan = Plan(c["L"], c["nlat"], c["nlon"], c["nu"], c["Omega"], precision=prec)
    full = plan.rhs(a).cpu().numpy()
    plan.set("CORIOLIS_SPLIT", 1)
    split = plan.rhs(a).cpu().numpy()
    e_split, e_full, e_diff = _rel(split, ref), _rel(full, ref), _rel(split, full)
    print(f"{prec}: split vs fp64 {e_split:.2e}, unsplit vs fp64 {e_full:.2e}, split vs unsplit {e_diff:.2e}")
    assert e_split <= tol and e_full <= tol and e_diff <= tol
