"""Batched ensemble (independent problems of uneven truncation and
viscosity in one graph-captured launch per RHS): each instance must get
exactly what a plan of its own gives, for the RHS and for adaptive steps."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from _parity import degree_order_errors
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


@pytest.mark.parametrize("precision,tol", [("fp32", 3e-5), ("bf16x3", 3e-5)])
def test_full_ensemble_rhs_matches_oracle_on_sampled_members(precision, tol):
    """The 256-member ensemble (L uniform over {63, 127, 255}, nu log-uniform
    in [1e-5, 1e-3]) in one batched RHS, as the ensemble benchmark runs it:
    two members of every truncation against the FP64 oracle's Galerkin RHS
    (Eq. (ode)); the rest must be finite."""
    from oracle.rhs import Problem, rhs_separable
    from paper_1009_3308_gb300 import Ensemble
    from seeded_inputs import ensemble
    mem = ensemble(256)
    ens = Ensemble([m["L"] for m in mem], [m["nu"] for m in mem], 1.0, precision=precision)
    for i, m in enumerate(mem):
        ens.set_alpha(i, _dev(m["alpha0"]))
    ens.rhs()
    torch.cuda.synchronize()
    picked = []
    for L in (63, 127, 255):
        idx = [i for i, m in enumerate(mem) if m["L"] == L]
        picked += [idx[0], idx[-1]]
    for i in picked:
        m = mem[i]
        ref = rhs_separable(Problem(m["L"], m["nlon"], m["nu"], m["Omega"]), m["alpha0"])
        got = ens.get(i, "F").cpu().numpy()
        err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
        assert err <= tol, (i, m["L"], err)
        prob = Problem(m["L"], m["nlon"], m["nu"], m["Omega"])
        eL, Lw, em, mw = degree_order_errors(got, ref, prob, m["alpha0"], floor=1e-2)
        assert eL <= 1e-3 and em <= 1e-3, (i, m["L"], eL, Lw, em, mw)
    for i in range(len(mem)):
        assert torch.isfinite(torch.view_as_real(ens.get(i, "F"))).all(), i


def test_advance_before_init_is_an_argument_error():
    from paper_1009_3308_gb300 import Ensemble, SphnseError
    ens = Ensemble([31, 31], [1e-3, 1e-3], 1.0)
    with pytest.raises(SphnseError, match="E_ARG"):
        ens.advance(1)
    ens.set_alpha(0, _dev(coefficients(31, 7, 0.1)))
    ens.init(0.0)
    assert len(ens.advance(0)) == 2


@pytest.mark.parametrize("precision", ["fp32", "bf16x3"])
def test_small_and_uneven_truncations_match_oracle(precision):
    """Truncations whose own smallest grid the batched kernels do not take
    (L = 1, 5, 31: fewer than 32 northern latitudes; L = 50: 3L + 2 = 152)
    run on a larger exact grid; F is the same (Eq. (M_choice))."""
    from oracle.rhs import Problem, rhs_separable
    from paper_1009_3308_gb300 import Ensemble
    Ls, nus = [31, 50, 5, 31, 1], [1e-3, 2e-4, 1e-2, 5e-4, 1e-2]
    ens = Ensemble(Ls, nus, 1.0, precision=precision)
    alphas = [coefficients(L, 300 + i, 0.1) * 3 for i, L in enumerate(Ls)]
    for i, a in enumerate(alphas):
        ens.set_alpha(i, _dev(a))
    ens.rhs()
    for i, (L, nu) in enumerate(zip(Ls, nus)):
        M = 3 * (L + 1) + (3 * (L + 1)) % 2
        ref = rhs_separable(Problem(L, M, nu, 1.0), alphas[i])
        got = ens.get(i, "F").cpu().numpy()
        assert np.linalg.norm(got - ref) <= 3e-5 * np.linalg.norm(ref), (i, L)
    ens.init(0.0)
    infos = ens.advance(3)
    assert all(x["t"] > 0.0 for x in infos)


def test_autotuned_synthesis_shape_gives_the_same_rhs():
    """The autotuner picks, per truncation, the instance-group width and
    pipeline depth of the tensor-core synthesis by timing; the shape does not
    change any instance's result."""
    from paper_1009_3308_gb300 import Ensemble
    Ls = [63] * 12 + [127] * 3
    nus = [1e-4 * (1 + i) for i in range(len(Ls))]
    alphas = [coefficients(L, 700 + i, 0.05) * 3 for i, L in enumerate(Ls)]
    out = {}
    for tune in (True, False):
        ens = Ensemble(Ls, nus, 1.0, precision="bf16x3", autotune=tune)
        for i, a in enumerate(alphas):
            ens.set_alpha(i, _dev(a))
        ens.rhs()
        out[tune] = ([ens.get(i, "F").cpu().numpy() for i in range(len(Ls))], ens.buckets())
    for got, ref in zip(out[True][0], out[False][0]):
        assert np.linalg.norm(got - ref) <= 1e-13 * np.linalg.norm(ref)
    tuned, fixed = out[True][1], out[False][1]
    assert [b["L"] for b in tuned] == [63, 127] and [b["instances"] for b in tuned] == [12, 3]
    for b in tuned:
        assert 1 <= b["group"] <= 9 and 4 <= b["stages"] <= 6 and b["cluster"] in (1, 2, 4) and b["syn_us"] > 0.0, b
    assert [b["group"] for b in fixed] == [6, 3] and all(b["syn_us"] == 0.0 for b in fixed)
    print(tuned)


@pytest.mark.parametrize("cluster", [2, 4])
def test_clustered_synthesis_gives_the_same_rhs(cluster):
    """CTAs of a cluster sharing every table tile by TMA multicast (each
    loads a slice of the latitudes for all of them): every instance's F
    equals the one of the synthesis without clusters, over 3 truncations
    and group counts that do and do not fill the last cluster."""
    from paper_1009_3308_gb300 import Ensemble
    Ls = [63] * 21 + [127] * 5 + [255] * 10
    nus = [1e-4 * (1 + 0.1 * i) for i in range(len(Ls))]
    alphas = [coefficients(L, 800 + i, 0.05) * 3 for i, L in enumerate(Ls)]
    out = {}
    for cs in (1, cluster):
        ens = Ensemble(Ls, nus, 1.0, precision="bf16x3", autotune=False, cluster=cs)
        for i, a in enumerate(alphas):
            ens.set_alpha(i, _dev(a))
        for _ in range(2):
            ens.rhs()
        out[cs] = [ens.get(i, "F").cpu().numpy() for i in range(len(Ls))]
        assert [b["cluster"] for b in ens.buckets()] == [cs] * 3
    for i, (got, ref) in enumerate(zip(out[cluster], out[1])):
        assert np.linalg.norm(got - ref) <= 1e-13 * np.linalg.norm(ref), i
