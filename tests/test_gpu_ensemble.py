"""Batched ensemble (independent problems of uneven truncation and
viscosity in one graph-captured launch per RHS): each instance must get
exactly what a plan of its own gives, for the RHS and for adaptive steps."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from seeded_inputs import coefficients

pytestmark = pytest.mark.gpu


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.complex128)).cuda()


LS = [63, 127, 63, 127, 255, 63]
NUS = [1e-3, 3e-4, 1e-5, 1e-4, 2e-5, 5e-4]


def _ensemble():
    from paper_1009_3308_gb300 import Ensemble
    ens = Ensemble(LS, NUS, 1.0)
    alphas = [coefficients(L, 1000 + i, 0.05) * 3 for i, L in enumerate(LS)]
    for i, a in enumerate(alphas):
        ens.set_alpha(i, _dev(a))
    return ens, alphas


def _single(L, nu):
    from paper_1009_3308_gb300 import Plan
    M = 3 * (L + 1)
    return Plan(L, M // 2, M, nu, 1.0, precision="fp32")


def test_ensemble_rhs_equals_single_instance():
    ens, alphas = _ensemble()
    ens.rhs()
    for i, (L, nu) in enumerate(zip(LS, NUS)):
        ref = _single(L, nu).rhs(_dev(alphas[i])).cpu().numpy()
        got = ens.get(i, "F").cpu().numpy()
        assert np.linalg.norm(got - ref) <= 1e-13 * np.linalg.norm(ref), i


def test_ensemble_steps_equal_independent_integrators():
    from paper_1009_3308_gb300 import Integrator
    ens, alphas = _ensemble()
    rt, at = 1e-6, 1e-10
    ens.set("RTOL", rt)
    ens.set("ATOL", at)
    ens.init(0.0)
    integs = []
    for i, (L, nu) in enumerate(zip(LS, NUS)):
        p = _single(L, nu)
        p.set("RTOL", rt)
        p.set("ATOL", at)
        integs.append((p, Integrator(p, _dev(alphas[i]))))
    for s in range(12):
        infos = ens.step()
        for i, (p, it) in enumerate(integs):
            ref = it.step()
            assert infos[i]["order"] == ref["order"], (s, i)
            assert abs(infos[i]["h"] - ref["h"]) <= 1e-12 * ref["h"], (s, i)
    for i, (p, it) in enumerate(integs):
        ref = it.alpha.cpu().numpy()
        got = ens.get(i).cpu().numpy()
        assert np.linalg.norm(got - ref) <= 1e-12 * np.linalg.norm(ref), i


@pytest.mark.parametrize("precision", ["fp32", "bf16x3"])
def test_ensemble_advance_equals_independent_integrators(precision):
    """sphnse_ensemble_advance: every instance takes its 15 steps at its own
    pace in asynchronous rounds and ends where an integrator of its own ends
    (same per-step decisions, so the same final time, order and state)."""
    from paper_1009_3308_gb300 import Ensemble, Integrator, Plan
    ens = Ensemble(LS, NUS, 1.0, precision=precision)
    alphas = [coefficients(L, 1000 + i, 0.05) * 3 for i, L in enumerate(LS)]
    for i, a in enumerate(alphas):
        ens.set_alpha(i, _dev(a))
    rt, at = 1e-6, 1e-10
    ens.set("RTOL", rt)
    ens.set("ATOL", at)
    ens.init(0.0)
    nsteps = 15
    infos = ens.advance(nsteps)
    for i, (L, nu) in enumerate(zip(LS, NUS)):
        M = 3 * (L + 1)
        p = Plan(L, M // 2, M, nu, 1.0, precision=precision)
        p.set("RTOL", rt)
        p.set("ATOL", at)
        it = Integrator(p, _dev(alphas[i]))
        refs = [it.step() for _ in range(nsteps)]
        last = refs[-1]
        assert infos[i]["order"] == last["order"], i
        assert abs(infos[i]["t"] - last["t"]) <= 1e-12 * last["t"], i
        assert infos[i]["rhs_evals"] == sum(r["rhs_evals"] for r in refs), i
        assert infos[i]["rejections"] == sum(r["rejections"] for r in refs), i
        ref = it.alpha.cpu().numpy()
        got = ens.get(i).cpu().numpy()
        assert np.linalg.norm(got - ref) <= 1e-12 * np.linalg.norm(ref), i
