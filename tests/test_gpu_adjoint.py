"""GPU adjoint (A11): J(alpha)^T, the reverse NDF step, the objective
gradient and the autograd wrapper, checked against the oracle's independent
tangent-linear model (dot-product identities <J v, w> = <v, J^T w>) and
against central finite differences of the GPU forward map (frozen
controller)."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle.ndf import NDF
from oracle.rhs import Problem, rhs_separable
from oracle.tlm import ReplayTLM, objective as obj_oracle, objective_tlm, rhs_tlm
from seeded_inputs import coefficients, random_packed, workload

pytestmark = pytest.mark.gpu


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.complex128)).cuda()


def _rdot(a, b):
    """real inner product of packed complex vectors (real components)"""
    return float(np.sum(a.real * b.real + a.imag * b.imag))


def _plan(L, nlon, nu, Om, precision="fp64"):
    from paper_1009_3308_gb300 import Plan
    return Plan(L, nlon // 2, nlon, nu, Om, precision=precision)


@pytest.mark.parametrize("L,nlon", [(7, 24), (15, 48), (31, 96), (63, 192)])
def test_rhs_adjoint_dot_product(L, nlon):
    nu, Om = 2e-3, 1.2
    prob = Problem(L, nlon, nu, Om)
    plan = _plan(L, nlon, nu, Om)
    a = coefficients(L, 10 + L, 0.05) * 5
    v = random_packed(L, 20 + L)
    w = random_packed(L, 30 + L)
    Jv = rhs_tlm(prob, a, v)
    JTw, nub = plan.rhs_adjoint(_dev(a), _dev(w), want_nu=True)
    JTw = JTw.cpu().numpy()
    lhs, rhs = _rdot(Jv, w), _rdot(v, JTw)
    assert abs(lhs - rhs) <= 1e-12 * np.linalg.norm(Jv) * np.linalg.norm(w), (lhs, rhs)
    # nu derivative: <w, dF/dnu> = -<w, lambda alpha>
    assert abs(nub + _rdot(w, prob.lam * a)) <= 1e-12 * abs(_rdot(w, prob.lam * a))


def test_objective_value_and_gradient():
    L, nlon = 31, 96
    prob = Problem(L, nlon, 1e-3, 1.0)
    plan = _plan(L, nlon, 1e-3, 1.0)
    a = coefficients(L, 5, 0.05)
    tgt = coefficients(L, 55, 0.05)
    lo, hi = math.radians(30), math.radians(60)
    J, g = plan.objective(_dev(a), _dev(tgt), lo, hi)
    assert abs(J - obj_oracle(prob, a, tgt, lo, hi)) <= 1e-12 * abs(J)
    g = g.cpu().numpy()
    for seed in range(3):
        v = random_packed(L, 700 + seed)
        ref = objective_tlm(prob, a, v, tgt, lo, hi)
        assert abs(_rdot(g, v) - ref) <= 1e-11 * (abs(ref) + np.linalg.norm(g) * np.linalg.norm(v) * 1e-3)


SCHED = [(2e-2, 1), (2e-2, 2), (3e-2, 2), (3e-2, 3), (2.5e-2, 3), (2.5e-2, 4), (4e-2, 5), (3e-2, 4)]


def test_trajectory_gradient_matches_oracle_tlm():
    """<grad_{alpha0} (w . alpha_T), v> + grad_nu dnu equals the oracle's
    tangent-linear directional derivative of the replayed trajectory."""
    from paper_1009_3308_gb300.adjoint import trajectory
    L, nlon, nu, Om = 15, 48, 5e-3, 1.0
    prob = Problem(L, nlon, nu, Om)
    plan = _plan(L, nlon, nu, Om)
    a0 = coefficients(L, 7, 0.1) * 5
    h0 = 2e-2
    w = random_packed(L, 8)
    a0r = torch.view_as_real(_dev(a0)).clone().requires_grad_(True)
    nut = torch.tensor(nu, dtype=torch.float64, requires_grad=True)
    aT = trajectory(plan, a0r, nut, SCHED, h0, checkpoint=3)
    loss = (aT * torch.view_as_real(_dev(w))).sum()
    loss.backward()
    g = torch.view_as_complex(a0r.grad).cpu().numpy()
    gnu = float(nut.grad)
    nd = NDF(lambda t, y: rhs_separable(prob, y), -prob.nu * prob.lam + 2j * Om * prob.ms / prob.lam, 0.0,
             a0, rtol=1e-6, atol=1e-9, h0=h0)
    for seed, dnu in ((1, 0.0), (2, 0.4), (3, -0.7)):
        v = random_packed(L, 100 + seed)
        nd2 = NDF(nd.rhs, nd.jdiag, 0.0, a0, rtol=1e-6, atol=1e-9, h0=h0)
        tl = ReplayTLM(prob, nd2, v, dnu)
        for h, k in SCHED:
            tl.step(h, k)
        ref = _rdot(w, tl.dy)
        got = _rdot(g, v) + gnu * dnu
        assert abs(got - ref) <= 1e-9 * (abs(ref) + 1e-30), (seed, got, ref)
    # the forward value is the oracle's replay
    ndf = NDF(nd.rhs, nd.jdiag, 0.0, a0, rtol=1e-6, atol=1e-9, h0=h0)
    for h, k in SCHED:
        ndf.replay_step(h, k)
    aTn = torch.view_as_complex(aT.detach()).cpu().numpy()
    assert np.linalg.norm(aTn - ndf.y) <= 1e-11 * np.linalg.norm(ndf.y)


def _fd_check(plan, a0, nu, sched, h0, tgt, lo, hi, ndir, seed0, eps=1e-6, checkpoint=20):
    from paper_1009_3308_gb300.adjoint import objective, trajectory
    a0r = torch.view_as_real(_dev(a0)).clone().requires_grad_(True)
    nut = torch.tensor(nu, dtype=torch.float64, requires_grad=True)
    J = objective(plan, trajectory(plan, a0r, nut, sched, h0, checkpoint=checkpoint), tgt, lo, hi)
    J.backward()
    g = torch.view_as_complex(a0r.grad).cpu().numpy()
    gnu = float(nut.grad)

    def Jof(a, nuv):
        with torch.no_grad():
            ar = torch.view_as_real(_dev(a)).clone()
            out = objective(plan, trajectory(plan, ar, torch.tensor(nuv, dtype=torch.float64), sched, h0,
                                             checkpoint=checkpoint), tgt, lo, hi)
        return float(out)
    errs = []
    scale = np.linalg.norm(a0)
    for d in range(ndir):
        v = random_packed(plan.L, seed0 + d)
        v = v / np.linalg.norm(v) * scale
        dnu = 0.1 * nu if d % 4 == 0 else 0.0
        fd = (Jof(a0 + eps * v, nu + eps * dnu) - Jof(a0 - eps * v, nu - eps * dnu)) / (2 * eps)
        ad = _rdot(g, v) + gnu * dnu
        errs.append(abs(fd - ad) / max(abs(fd), 1e-300))
    return max(errs), g, gnu


def test_gradient_vs_finite_differences_L31():
    from paper_1009_3308_gb300.adjoint import adaptive_schedule
    L, nlon, nu, Om = 31, 96, 1e-3, 1.0
    plan = _plan(L, nlon, nu, Om)
    plan.set("RTOL", 1e-6)
    plan.set("ATOL", 1e-10)
    a0 = coefficients(L, 5, 0.05) * 3
    tgt = _dev(coefficients(L, 55, 0.05))
    _, sched, h0 = adaptive_schedule(plan, _dev(a0), 25)
    err, _, _ = _fd_check(plan, a0, nu, sched, h0, tgt, math.radians(30), math.radians(60), 6, 900,
                          checkpoint=7)
    assert err <= 1e-6, err


def test_adjoint_workload_L255_full_size():
    """Adjoint workload: L = 255 on 384 x 768, 200 steps, checkpoints every 20,
    gradient of band energy + misfit w.r.t. alpha0 and nu against central
    finite differences (h = 1e-6) on 16 random directions (FP64); and the
    FP32-contraction gradient against the FP64 one."""
    from paper_1009_3308_gb300.adjoint import adaptive_schedule
    w = workload("adjoint")
    c = w["config"]
    plan = _plan(c["L"], c["nlon"], c["nu"], c["Omega"])
    plan.set("RTOL", c["rtol"])
    plan.set("ATOL", 1e-3 * c["rtol"] * float(np.max(np.abs(w["alpha0"]))))
    a0 = w["alpha0"]
    tgt = _dev(w["target"])
    _, sched, h0 = adaptive_schedule(plan, _dev(a0), c["steps"])
    lo, hi = math.radians(30), math.radians(60)
    err, g64, gnu64 = _fd_check(plan, a0, c["nu"], sched, h0, tgt, lo, hi, 16, 1200, checkpoint=c["checkpoint"])
    assert err <= 2e-5, err
    plan.set_precision("fp32")
    from paper_1009_3308_gb300.adjoint import objective, trajectory
    a0r = torch.view_as_real(_dev(a0)).clone().requires_grad_(True)
    nut = torch.tensor(c["nu"], dtype=torch.float64, requires_grad=True)
    J = objective(plan, trajectory(plan, a0r, nut, sched, h0, checkpoint=c["checkpoint"]), tgt, lo, hi)
    J.backward()
    g32 = torch.view_as_complex(a0r.grad).cpu().numpy()
    assert np.linalg.norm(g32 - g64) <= 1e-3 * np.linalg.norm(g64)
