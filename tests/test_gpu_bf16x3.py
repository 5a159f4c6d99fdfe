"""BF16 hi + lo split-precision Legendre contractions on tcgen05 tensor
cores (FP32 accumulation), checked against the FP64 oracle.

Error budget: each operand is split as x = hi + lo with hi, lo in BF16
(8-bit significands), so |x - hi - lo| <= 2^-17 |x|; the products keep all
four terms hi*hi + hi*lo + lo*hi + lo*lo; FP32 accumulation adds ~2^-24
sqrt(n).  Per contraction output the relative error is ~1e-5 of the sum of
|terms|; the tests take 3e-5 on F (norm), 1e-5 per grid field and 1e-4 on
the state after 500 replayed steps at L = 511, and state the measured
errors."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from _parity import degree_order_errors
from oracle.rhs import Problem, rhs_separable
from seeded_inputs import coefficients, workload

pytestmark = pytest.mark.gpu


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.complex128)).cuda()


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("L,nlon,nu,Om,decay", [(31, 96, 1e-2, 1.0, 0.3), (63, 192, 1e-3, 1.0, 0.1),
                                                (127, 384, 1e-4, 1.0, 0.05), (255, 768, 1e-4, 1.0, 0.05)])
def test_rhs_bf16x3_matches_oracle(L, nlon, nu, Om, decay):
    from paper_1009_3308_gb300 import Plan
    prob = Problem(L, nlon, nu, Om)
    a = coefficients(L, 400 + L, decay) * 3.0
    ref = rhs_separable(prob, a)
    plan = Plan(L, nlon // 2, nlon, nu, Om, precision="bf16x3")
    got = plan.rhs(_dev(a)).cpu().numpy()
    err = _rel(got, ref)
    eL, Lw, em, mw = degree_order_errors(got, ref, prob, a, floor=1e-2)
    print(f"L={L} bf16x3 rel err {err:.3e}; per degree {eL:.2e} (L={Lw}), per order {em:.2e} (m={mw})")
    assert err <= 3e-5, err
    assert eL <= 1e-3 and em <= 1e-3, (eL, Lw, em, mw)
    assert plan.sync() == 0


def test_rhs_bf16x3_L511_vs_fp64():
    from paper_1009_3308_gb300 import Plan
    w = workload("L511")
    c = w["config"]
    plan = Plan(c["L"], c["nlat"], c["nlon"], c["nu"], c["Omega"])
    a = _dev(w["alpha0"])
    f64 = plan.rhs(a).cpu().numpy()
    plan.set_precision("bf16x3")
    fb = plan.rhs(a).cpu().numpy()
    err = _rel(fb, f64)
    print(f"L=511 bf16x3 vs fp64 rel err {err:.3e}")
    assert err <= 3e-5, err
    assert plan.sync() == 0


def test_ensemble_bf16x3_groups_match_fp64_plans():
    """Batched tensor-core synthesis: 23 instances at L = 63 (three instance
    groups sharing each table tile), three at 127 and two at 255; every
    instance's F against a plan of its own in FP64."""
    from paper_1009_3308_gb300 import Ensemble, Plan
    Ls = [63] * 23 + [127] * 3 + [255] * 2
    nus = [1e-3 * (0.9 ** i) for i in range(len(Ls))]
    ens = Ensemble(Ls, nus, 1.0, precision="bf16x3")
    alphas = [coefficients(L, 2000 + i, 0.05) * 3 for i, L in enumerate(Ls)]
    for i, a in enumerate(alphas):
        ens.set_alpha(i, _dev(a))
    ens.rhs()
    worst = 0.0
    for i, (L, nu) in enumerate(zip(Ls, nus)):
        M = 3 * (L + 1)
        ref = Plan(L, M // 2, M, nu, 1.0).rhs(_dev(alphas[i])).cpu().numpy()
        got = ens.get(i, "F").cpu().numpy()
        err = _rel(got, ref)
        worst = max(worst, err)
        assert err <= 3e-5, (i, L, err)
    print(f"ensemble bf16x3 worst rel err {worst:.3e}")


def test_grid_fields_and_projection_bf16x3_per_field():
    """Per field at L = 511: zeta, u_theta, u_phi on the grid (tensor-core
    synthesis) and the projection of a tangential field (tensor-core
    analysis), against the FP64 path."""
    from paper_1009_3308_gb300 import Plan
    w = workload("L511")
    c = w["config"]
    a = _dev(w["alpha0"])
    plan = Plan(c["L"], c["nlat"], c["nlon"], c["nu"], c["Omega"])
    ref = [x.cpu().numpy() for x in plan.grid_fields(a)]
    pref = plan.project(*[torch.from_numpy(r).cuda() for r in ref[1:]]).cpu().numpy()
    plan.set_precision("bf16x3")
    got = [x.cpu().numpy() for x in plan.grid_fields(a)]
    pgot = plan.project(*[torch.from_numpy(r).cuda() for r in ref[1:]]).cpu().numpy()
    errs = {n: _rel(g, r) for n, g, r in zip(("zeta", "u_theta", "u_phi"), got, ref)}
    errs["projection"] = _rel(pgot, pref)
    print("bf16x3 per field:", {k: f"{v:.2e}" for k, v in errs.items()})
    # u_phi at m = 0 is summed over the order-1 table (d/dtheta Pt_K^0 =
    # sqrt(K (K+1)) Pt_K^1); through the degree-shift relation divided by
    # sin(theta) it measured 2.5e-5, from cancellation near the poles
    bounds = {"zeta": 1e-5, "u_theta": 1e-5, "u_phi": 1e-5, "projection": 1e-5}
    for k, v in errs.items():
        assert v <= bounds[k], (k, v)


def test_state_after_500_replayed_steps_bf16x3_vs_fp64():
    """The mixed workload's 500 steps (rtol 1e-6): record the adaptive (h,
    order) sequence of the BF16X3 run, replay it in BF16X3 and in FP64 (each
    corrector solved to its convergence floor) and compare the final states."""
    from paper_1009_3308_gb300 import Integrator, Plan
    w = workload("L511")
    c = w["config"]
    a0 = _dev(w["alpha0"])
    atol = 1e-3 * c["rtol"] * float(abs(w["alpha0"]).max())

    def make(prec):
        p = Plan(c["L"], c["nlat"], c["nlon"], c["nu"], c["Omega"], precision=prec)
        p.set("RTOL", c["rtol"])
        p.set("ATOL", atol)
        return p, Integrator(p, a0.clone())

    _, run = make("bf16x3")
    sched = []
    for _ in range(500):
        info = run.step()
        sched.append((info["h"], info["order"]))
    states = {}
    for prec in ("bf16x3", "fp64"):
        _, it = make(prec)
        for h, k in sched:
            it.replay_step(h, k)
        states[prec] = it.alpha.cpu().numpy()
    err = _rel(states["bf16x3"], states["fp64"])
    drift = _rel(run.alpha.cpu().numpy(), states["fp64"])
    print(f"500 replayed steps: bf16x3 vs fp64 state rel err {err:.3e} (adaptive run vs fp64 replay {drift:.3e}),"
          f" t = {sum(h for h, _ in sched):.4g}")
    assert err <= 1e-4, err


@pytest.mark.parametrize("prec", ["fp64", "fp32", "bf16x3"])
def test_zero_state_gives_the_forcing_exactly(prec):
    """Degenerate case: alpha = 0 has no nonlinear, Coriolis or viscous term,
    so F = fhat bit for bit in every precision (L = 511 workload grid)."""
    from paper_1009_3308_gb300 import Plan
    w = workload("L511")
    c = w["config"]
    f = coefficients(c["L"], 4242, 0.02)
    plan = Plan(c["L"], c["nlat"], c["nlon"], c["nu"], c["Omega"], precision=prec)
    got = plan.rhs(_dev(np.zeros_like(f)), forcing=_dev(f)).cpu().numpy()
    np.testing.assert_array_equal(got, f)


@pytest.mark.parametrize("prec,split", [("fp32", 0), ("bf16x3", 0), ("bf16x3", 1)])
def test_forced_state_matches_oracle(prec, split):
    """A nonzero state with a nonzero forcing on every coefficient (Eq.
    (ode): F = fhat - nu lam alpha - N), with and without the split Coriolis
    term (Eq. (Coriolis_ZLm)): the FP32 update adds the forcing in FP64, and
    here both parts are of the same size. L = 63 on 96 x 192 (tensor-core
    grid), against the FP64 oracle."""
    from paper_1009_3308_gb300 import Plan
    L, nlon, nu, Om = 63, 192, 1e-3, 1.0
    prob = Problem(L, nlon, nu, Om)
    a = coefficients(L, 777, 0.1) * 3.0
    ref0 = rhs_separable(prob, a)
    f = coefficients(L, 778, 0.1) * (np.linalg.norm(ref0) / np.linalg.norm(coefficients(L, 778, 0.1)))
    ref = rhs_separable(prob, a, forcing=f)
    plan = Plan(L, nlon // 2, nlon, nu, Om, precision=prec)
    if split:
        plan.set("CORIOLIS_SPLIT", 1)
    got = plan.rhs(_dev(a), forcing=_dev(f)).cpu().numpy()
    err = _rel(got, ref)
    # the forcing itself passes unchanged: F - fhat against the unforced oracle
    err0 = _rel(got - f, ref0)
    print(f"{prec} split={split}: forced rel err {err:.2e}, unforced part {err0:.2e}")
    assert err <= 3e-5 and err0 <= 3e-5, (err, err0)
    assert plan.sync() == 0


@pytest.mark.parametrize("L,nlon", [(5, 18), (127, 768)])
def test_bf16x3_plan_off_the_tensor_core_grid(L, nlon):
    """A BF16X3 plan whose grid the tensor-core kernels do not take (odd
    nlat) runs the FP32 kernels; an oversampled grid (M = 6 (N + 1)) runs the
    tensor-core kernels with 192 northern nodes: both within the mixed bound
    against the oracle."""
    from paper_1009_3308_gb300 import Plan
    prob = Problem(L, nlon, 1e-3, 1.0)
    a = coefficients(L, 500 + L, 0.05) * 3.0
    ref = rhs_separable(prob, a)
    got = Plan(L, nlon // 2, nlon, 1e-3, 1.0, precision="bf16x3").rhs(_dev(a)).cpu().numpy()
    err = _rel(got, ref)
    print(f"L={L} nlon={nlon} bf16x3 plan rel err {err:.2e}")
    assert err <= 3e-5, err

