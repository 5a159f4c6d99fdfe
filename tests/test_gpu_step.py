"""GPU NDF time step (Sec. 4.2, Eq. (ode_disc)) against the oracle's NDF.

* replay: a step-size/order schedule fixed by the test is applied by both
  sides; states must agree to FP64 rounding accumulated over the steps;
* adaptive: both controllers run independently from the same inputs and
  must take the same orders, step sizes (to rounding) and states;
* closed form: single-degree data evolve as exp((-nu lambda + 2 i Omega m /
  lambda) t);
* error paths: a non-finite state is reported, not integrated.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle.ndf import NDF
from oracle.rhs import Problem, rhs_separable
from seeded_inputs import coefficients, random_packed, workload

pytestmark = pytest.mark.gpu


def _jd(prob):
    return -prob.nu * prob.lam + 2j * prob.Omega * prob.ms / prob.lam


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.complex128)).cuda()


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _l31():
    from paper_1009_3308_gb300 import Plan
    w = workload("L31")
    c = w["config"]
    prob = Problem(c["L"], c["nlon"], c["nu"], c["Omega"])
    plan = Plan(c["L"], c["nlat"], c["nlon"], c["nu"], c["Omega"])
    return w, c, prob, plan


SCHED = [(1e-3, 1), (1e-3, 2), (1.5e-3, 2), (1.5e-3, 3), (2e-3, 3), (2e-3, 4), (2e-3, 5), (3e-3, 5),
         (2.5e-3, 4), (2.5e-3, 3), (4e-3, 2), (4e-3, 1)]


def test_replay_matches_oracle():
    from paper_1009_3308_gb300 import Integrator
    w, c, prob, plan = _l31()
    a0, f = w["alpha0"] * 20.0, w["forcing"]
    rt, at = 1e-8, 1e-12
    plan.set("RTOL", rt)
    plan.set("ATOL", at)
    nd = NDF(lambda t, y: rhs_separable(prob, y, f), _jd(prob), 0.0, a0, rtol=rt, atol=at, h0=1e-3)
    integ = Integrator(plan, _dev(a0), h0=1e-3, forcing=_dev(f))
    for h, k in SCHED:
        nd.replay_step(h, k)
        integ.replay_step(h, k)
        got = integ.alpha.cpu().numpy()
        assert _rel(got, nd.y) <= 1e-11, (h, k, _rel(got, nd.y))
    np.testing.assert_allclose(integ.dif.cpu().numpy()[:6], nd.dif[:6], rtol=0,
                               atol=1e-10 * np.max(np.abs(nd.dif[:6])))


def test_adaptive_controller_matches_oracle_L31():
    """The L = 31 workload at its stated length (100 adaptive steps, rtol
    1e-8, steady forcing): both adaptive integrators take the same decisions,
    and alpha(t_100) agrees."""
    from paper_1009_3308_gb300 import Integrator
    w, c, prob, plan = _l31()
    a0, f = w["alpha0"], w["forcing"]
    rt = c["rtol"]
    at = 1e-3 * rt * float(np.max(np.abs(a0)))
    plan.set("RTOL", rt)
    plan.set("ATOL", at)
    nd = NDF(lambda t, y: rhs_separable(prob, y, f), _jd(prob), 0.0, a0, rtol=rt, atol=at)
    integ = Integrator(plan, _dev(a0), forcing=_dev(f))
    assert abs(integ.h0 - nd.h) <= 1e-12 * nd.h
    for s in range(c["steps"]):
        io = nd.step()
        ig = integ.step()
        assert ig["order"] == io["order"], (s, ig, io)
        # h_new = h (rtol / err)^(1/(k+1)) with err a norm of d = alpha_{n+1} - alpha^(0),
        # a difference of nearly equal states: rounding-level differences in
        # F appear amplified (~1e-9 relative) in the chosen step sizes
        assert abs(ig["h"] - io["h"]) <= 1e-6 * io["h"], (s, ig["h"], io["h"])
        assert ig["rejections"] == io["rejections"]
    err = _rel(integ.alpha.cpu().numpy(), nd.y)
    print(f"L=31 after {c['steps']} adaptive steps: t = {nd.t:.6g}, alpha rel err {err:.2e}")
    assert err <= 1e-7
    assert abs(integ.t - nd.t) <= 1e-6 * nd.t


def test_rossby_haurwitz_on_gpu():
    from paper_1009_3308_gb300 import Integrator, Plan
    L, nlon, nu, Om = 63, 192, 1e-3, 1.0
    prob = Problem(L, nlon, nu, Om)
    a0 = np.where(prob.Ls == 10, random_packed(L, 3), 0)
    plan = Plan(L, nlon // 2, nlon, nu, Om)
    rt = 1e-8
    plan.set("RTOL", rt)
    plan.set("ATOL", 1e-3 * rt)
    integ = Integrator(plan, _dev(a0))
    for _ in range(30):
        integ.step()
    exact = a0 * np.exp(_jd(prob) * integ.t)
    assert np.max(np.abs(integ.alpha.cpu().numpy() - exact)) <= 100 * rt * np.max(np.abs(a0))


def test_nonfinite_state_is_reported():
    from paper_1009_3308_gb300 import Integrator, SphnseError
    w, c, prob, plan = _l31()
    a = w["alpha0"].copy()
    a[5] = np.nan
    integ = Integrator(plan, _dev(a), h0=1e-3)
    with pytest.raises(SphnseError, match="E_NONFINITE"):
        integ.step()


def test_step_argument_errors():
    from paper_1009_3308_gb300 import Integrator, SphnseError
    w, c, prob, plan = _l31()
    integ = Integrator(plan, _dev(w["alpha0"]), h0=1e-3)
    with pytest.raises(SphnseError, match="E_ARG"):
        integ.replay_step(1e-3, 7)
    with pytest.raises(SphnseError, match="E_ARG"):
        integ.replay_step(-1.0, 1)


def test_advance_equals_repeated_steps():
    """sphnse_advance(n) takes exactly the steps of n sphnse_step calls."""
    from paper_1009_3308_gb300 import Integrator
    w, c, prob, plan = _l31()
    a0, f = w["alpha0"], w["forcing"]
    plan.set("RTOL", c["rtol"])
    plan.set("ATOL", 1e-3 * c["rtol"] * float(np.max(np.abs(a0))))
    i1 = Integrator(plan, _dev(a0), forcing=_dev(f))
    ref = [i1.step() for _ in range(15)]
    i2 = Integrator(plan, _dev(a0), forcing=_dev(f))
    got = i2.advance(15)
    assert [g["h"] for g in got] == [r["h"] for r in ref]
    assert [g["order"] for g in got] == [r["order"] for r in ref]
    assert torch.equal(i1.alpha, i2.alpha)
