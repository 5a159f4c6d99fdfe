"""Pins of the oracle's tangent-linear model against central finite
differences of the oracle itself (RHS, frozen-controller NDF trajectory,
objective)."""
import numpy as np

from oracle.ndf import NDF
from oracle.rhs import Problem, rhs_separable
from oracle.tlm import ReplayTLM, objective, objective_tlm, rhs_tlm
from seeded_inputs import coefficients, random_packed


def test_rhs_tlm_vs_central_difference():
    prob = Problem(9, 30, 2e-3, 1.1)
    a = coefficients(9, 4, 0.1)
    v = random_packed(9, 5, 0.05)
    eps = 1e-5
    fd = (rhs_separable(prob, a + eps * v) - rhs_separable(prob, a - eps * v)) / (2 * eps)
    assert np.linalg.norm(rhs_tlm(prob, a, v) - fd) <= 1e-8 * np.linalg.norm(fd)
    # nu-derivative
    p2 = Problem(9, 30, 2e-3 + 1e-7, 1.1)
    p1 = Problem(9, 30, 2e-3 - 1e-7, 1.1)
    fdn = (rhs_separable(p2, a) - rhs_separable(p1, a)) / 2e-7
    dn = rhs_tlm(prob, a, np.zeros_like(a), 1.0)
    assert np.linalg.norm(dn - fdn) <= 1e-7 * np.linalg.norm(fdn)


def _run(prob, a0, schedule, h0):
    jd = -prob.nu * prob.lam + 2j * prob.Omega * prob.ms / prob.lam
    nd = NDF(lambda t, y: rhs_separable(prob, y), jd, 0.0, a0, rtol=1e-6, atol=1e-9, h0=h0)
    for h, k in schedule:
        nd.replay_step(h, k)
    return nd


def test_replay_tlm_vs_central_difference():
    N, M = 6, 22
    nu, Om = 5e-3, 1.0
    prob = Problem(N, M, nu, Om)
    a0 = coefficients(N, 7, 0.1) * 5
    v = random_packed(N, 8, 1.0)
    dnu = 0.3
    sched = [(0.02, 1), (0.02, 2), (0.03, 2), (0.03, 3), (0.025, 3), (0.025, 4), (0.04, 5), (0.03, 4)]
    h0 = 0.02
    eps = 1e-6
    jd = -prob.nu * prob.lam + 2j * prob.Omega * prob.ms / prob.lam
    nd = NDF(lambda t, y: rhs_separable(prob, y), jd, 0.0, a0, rtol=1e-6, atol=1e-9, h0=h0)
    tl = ReplayTLM(prob, nd, v, dnu)
    for h, k in sched:
        tl.step(h, k)
    plus = _run(Problem(N, M, nu + eps * dnu, Om), a0 + eps * v, sched, h0)
    minus = _run(Problem(N, M, nu - eps * dnu, Om), a0 - eps * v, sched, h0)
    fd = (plus.y - minus.y) / (2 * eps)
    assert np.linalg.norm(tl.dy - fd) <= 1e-7 * np.linalg.norm(fd)


def test_objective_tlm_vs_central_difference():
    prob = Problem(8, 28, 1e-3, 1.0)
    a = coefficients(8, 1, 0.1)
    tgt = coefficients(8, 2, 0.1)
    v = random_packed(8, 3)
    lo, hi = np.radians(30), np.radians(60)
    eps = 1e-6
    fd = (objective(prob, a + eps * v, tgt, lo, hi) - objective(prob, a - eps * v, tgt, lo, hi)) / (2 * eps)
    assert abs(objective_tlm(prob, a, v, tgt, lo, hi) - fd) <= 1e-8 * abs(fd)
