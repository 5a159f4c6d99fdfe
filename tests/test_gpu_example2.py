"""Sec. 5 Example 2 (N = 100, Omega = 1, nu = 1e-4, rtol 1e-3): the random
initial state of degree <= 20 driven by fhat_{3,0}(t).

Against the oracle: both adaptive integrators, given the forcing at the end
of each planned step, take the same orders, rejections and step sizes, and
reach the same state, from t = 0 and over the switch of fhat_{3,0} at t = 10.

The paper compares plots; the long-run checks take the properties it reports
in numbers:
- the initial small structures give way to larger ones (the energy centroid
  of U_75 moves to lower degrees);
- L^4 E(Phi_150(U_75), L) of the approximate inertial manifold
  (Eq. (eq:p-p)) decays exponentially in L (Sec. 6.2).
Integrated to t = 20 here; bench.py runs to t = 60."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle.ndf import NDF
from oracle.rhs import Problem, rhs_separable
from seeded_inputs import example2, example2_forcing_30

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("t0,nsteps", [(0.0, 40), (9.9, 60)])
def test_example2_steps_match_oracle(t0, nsteps):
    from paper_1009_3308_gb300 import Integrator, Plan
    N, nu, rtol = 100, 1e-4, 1e-3
    a0 = example2(N)
    atol = 1e-3 * rtol * float(np.abs(a0).max())
    plan = Plan(N, 162, 324, nu, 1.0)
    plan.set("RTOL", rtol)
    plan.set("ATOL", atol)
    prob = Problem(N, 324, nu, 1.0)
    fo = np.zeros(prob.n(), dtype=np.complex128)
    fo[2] = example2_forcing_30(t0)          # packed index of (L, m) = (3, 0)
    nd = NDF(lambda t, y: rhs_separable(prob, y, fo), -prob.nu * prob.lam + 2j * prob.ms / prob.lam, t0, a0,
             rtol=rtol, atol=atol)
    f = torch.from_numpy(fo.copy()).cuda()
    it = Integrator(plan, torch.from_numpy(a0).cuda(), t0=t0, forcing=f)
    assert abs(it.h0 - nd.h) <= 1e-12 * nd.h
    rej = 0
    for s in range(nsteps):
        fo[2] = example2_forcing_30(nd.t + nd.h)
        f[2] = example2_forcing_30(it.t + it.st.h)
        io = nd.step()
        ig = it.step()
        assert ig["order"] == io["order"] and ig["rejections"] == io["rejections"], (s, ig, io)
        assert abs(ig["h"] - io["h"]) <= 1e-6 * io["h"], (s, ig["h"], io["h"])
        rej += io["rejections"]
    err = float(np.linalg.norm(it.alpha.cpu().numpy() - nd.y) / np.linalg.norm(nd.y))
    print(f"Example 2 from t = {t0}: {nsteps} steps to t = {nd.t:.5f}, {rej} rejections, state rel err {err:.2e}")
    assert err <= 1e-7
    assert abs(it.t - nd.t) <= 1e-6 * nd.t
    if t0 > 0:
        assert nd.t > 10.0   # the stretch crosses the switch of the forcing


def test_example2_large_structures_and_inertial_manifold_decay():
    from paper_1009_3308_gb300 import Integrator, Plan
    N, N1, nu, rtol = 100, 75, 1e-4, 1e-3
    plan = Plan(N, 162, 324, nu, 1.0)
    plan.set("RTOL", rtol)
    a0 = example2(N)
    plan.set("ATOL", 1e-3 * rtol * float(np.abs(a0).max()))
    p2 = Plan(2 * N1, 243, 486, nu, 1.0)
    f = torch.zeros(plan.n_coeff, dtype=torch.complex128, device="cuda")
    f2 = torch.zeros(p2.n_coeff, dtype=torch.complex128, device="cuda")
    it = Integrator(plan, torch.from_numpy(a0).cuda(), forcing=f)
    L = np.arange(N1 + 1)

    def centroid(a):
        E = plan.energy_spectrum(a).cpu().numpy()[: N1 + 1]
        return float((L[1:] * E[1:]).sum() / E[1:].sum())

    c0 = centroid(it.alpha)
    for te in (10.0, 20.0):
        it.st.t_end = te
        while it.t < te * (1 - 1e-12):
            f[2] = example2_forcing_30(min(te, it.t + it.st.h))
            it.step()
        f2[2] = example2_forcing_30(te)
        phi = p2.inertial_manifold(N1, p2.resize(it.alpha, N, L_max=N1), f2)
        Ep = p2.energy_spectrum(phi).cpu().numpy()
        Lp = np.arange(N1 + 1, 2 * N1 + 1)
        y = np.log(Lp ** 4 * Ep[N1 + 1:])
        slope = np.polyfit(Lp, y, 1)[0]
        drop = y[:5].mean() - y[-5:].mean()
        print(f"t={te}: centroid {centroid(it.alpha):.3f} (t=0: {c0:.3f}); log L^4 E(Phi): slope {slope:.3f} per degree, "
              f"{drop / math.log(10):.1f} decades from L = 76 to 150")
        assert slope < -0.1 and drop > 10 * math.log(10), (te, slope, drop)
    assert centroid(it.alpha) < 0.6 * c0
    assert math.isfinite(float(torch.linalg.vector_norm(it.alpha).item()))
