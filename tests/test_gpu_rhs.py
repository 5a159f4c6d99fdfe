"""GPU parity of the RHS F (Eq. (ode)) and its transforms against the FP64
oracle, through the C ABI.

Tolerances: FP64 path ||F_gpu - F_oracle||_2 / ||F_oracle||_2 <= 1e-12
(every step is FP64 on both sides; differences are rounding order only).
FP32 path: FP32 tables/contractions/FFTs with FP32 accumulation over at most
~L/2 + 1 terms and log2(M) FFT stages: per-field relative error bounded by
~(L/2 + 2 log2 M) * 6e-8 in norm; the tests take 3e-5 for F and 1e-5 per grid
field."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from _parity import degree_order_errors
from oracle.rhs import Problem, project, rhs_separable, synthesize
from seeded_inputs import coefficients, random_packed, workload

pytestmark = pytest.mark.gpu

CASES = [
    # (L, nlon, nu, Omega, decay)  several tiles, ragged tails, odd nlat
    (1, 6, 1e-2, 1.0, 0.1),        # smallest plan
    (5, 18, 1e-2, 0.7, 0.1),       # nlat = 9 (odd: equator node)
    (7, 24, 1e-2, 1.0, 0.1),
    (17, 54, 3e-3, 1.3, 0.1),      # nlat = 27 (odd)
    (31, 96, 1e-2, 1.0, 0.3),      # the L = 31 workload grid
    (63, 192, 1e-3, 1.0, 0.05),    # two p-tiles? (nh = 48) ragged j-tiles
    (127, 384, 1e-4, 1.0, 0.05),   # nh = 96
]


def _plan(L, nlon, nu, Om, precision="fp64"):
    from paper_1009_3308_gb300 import Plan
    return Plan(L, nlon // 2, nlon, nu, Om, precision=precision)


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.complex128)).cuda()


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("L,nlon,nu,Om,decay", CASES)
def test_rhs_fp64_matches_oracle(L, nlon, nu, Om, decay):
    prob = Problem(L, nlon, nu, Om)
    a = coefficients(L, 100 + L, decay) * 3.0
    f = random_packed(L, 200 + L, 1e-3)
    ref = rhs_separable(prob, a, f)
    plan = _plan(L, nlon, nu, Om)
    got = plan.rhs(_dev(a), _dev(f)).cpu().numpy()
    assert _rel(got, ref) <= 1e-12, _rel(got, ref)
    # nonlinear part per degree and per order, above 1e-6 of the largest degree
    eL, Lw, em, mw = degree_order_errors(got, ref, prob, a, f, floor=1e-6)
    assert eL <= 1e-8 and em <= 1e-8, (eL, Lw, em, mw)
    # no forcing
    got0 = plan.rhs(_dev(a)).cpu().numpy()
    assert _rel(got0, rhs_separable(prob, a)) <= 1e-12


@pytest.mark.parametrize("L,nlon", [(7, 24), (31, 96), (63, 192)])
def test_grid_fields_and_projection_fp64(L, nlon):
    prob = Problem(L, nlon, 1e-3, 1.0)
    a = random_packed(L, 7)
    plan = _plan(L, nlon, 1e-3, 1.0)
    z, ut, up = (t.cpu().numpy() for t in plan.grid_fields(_dev(a)))
    rz, rut, rup = synthesize(prob, a)
    for got, ref in ((z, rz), (ut, rut), (up, rup)):
        assert _rel(got, ref) <= 1e-13
    pr = plan.project(torch.from_numpy(rut).cuda(), torch.from_numpy(rup).cuda()).cpu().numpy()
    assert _rel(pr, project(prob, rut, rup)) <= 1e-13
    assert _rel(pr, a) <= 1e-13   # round trip (Eq. (disc_proj_prop1))


@pytest.mark.parametrize("L,nlon,nu,Om,decay", [c for c in CASES if c[0] >= 5])
def test_rhs_fp32_matches_oracle(L, nlon, nu, Om, decay):
    prob = Problem(L, nlon, nu, Om)
    a = coefficients(L, 300 + L, decay) * 3.0
    ref = rhs_separable(prob, a)
    plan = _plan(L, nlon, nu, Om, "fp32")
    got = plan.rhs(_dev(a)).cpu().numpy()
    assert _rel(got, ref) <= 3e-5, _rel(got, ref)
    eL, Lw, em, mw = degree_order_errors(got, ref, prob, a, floor=1e-2)
    assert eL <= 1e-3 and em <= 1e-3, (eL, Lw, em, mw)


def test_rhs_invariants_fp64_L255_full_size():
    """L = 255 on 384 x 768 (the FP64 workload): full oracle parity and the
    energy/enstrophy invariants of Thm 4.1 on the GPU output."""
    w = workload("L255")
    c = w["config"]
    prob = Problem(c["L"], c["nlon"], c["nu"], c["Omega"])
    a = w["alpha0"]
    plan = _plan(c["L"], c["nlon"], c["nu"], c["Omega"])
    got = plan.rhs(_dev(a)).cpu().numpy()
    ref = rhs_separable(prob, a)
    assert _rel(got, ref) <= 1e-12, _rel(got, ref)
    eL, Lw, em, mw = degree_order_errors(got, ref, prob, a, floor=1e-6)
    assert eL <= 1e-8 and em <= 1e-8, (eL, Lw, em, mw)
    Nn = -(got + prob.nu * prob.lam * a)
    s = np.where(prob.ms == 0, 1.0, 2.0)
    e = np.sum(s * np.conj(a) * Nn).real / (np.linalg.norm(a) * np.linalg.norm(Nn))
    z = np.sum(s * prob.lam * np.conj(a) * Nn).real / (np.linalg.norm(prob.lam * a) * np.linalg.norm(Nn))
    assert abs(e) < 1e-12 and abs(z) < 1e-12


def test_rhs_L511_full_size_properties():
    """L = 511 on 768 x 1536: the sizes the benchmark times.  Checks that hold
    at any size: single-degree data give the closed form (Eq. (Coriolis_ZLm)),
    the energy and enstrophy invariants, and FP32 vs FP64 agreement."""
    w = workload("L511")
    c = w["config"]
    L, nlon = c["L"], c["nlon"]
    plan = _plan(L, nlon, c["nu"], c["Omega"])
    Ls, ms = np.array([], int), np.array([], int)
    from oracle.layout import packed_degrees_orders
    Ls, ms = packed_degrees_orders(L)
    lam = Ls * (Ls + 1.0)
    # single degree L0 = 300: only the diagonal terms survive; the gradient
    # part of the product cancels in the projection, so the bound is relative
    # to the quadrature L2 norm of W = (zeta + 2 Omega cos) xhat x u
    b = np.where(Ls == 300, random_packed(L, 77), 0)
    got = plan.rhs(_dev(b)).cpu().numpy()
    expect = (-c["nu"] * lam + 2j * c["Omega"] * ms / lam) * b
    z, ut, up = (t.cpu().numpy() for t in plan.grid_fields(_dev(b)))
    th, x, s, wq = (t.numpy() for t in plan.nodes())
    q = z + 2 * c["Omega"] * x[:, None]
    normW = np.sqrt(np.sum((2 * np.pi / nlon) * wq[:, None] * q * q * (ut * ut + up * up)))
    assert np.linalg.norm(got - expect) <= 1e-13 * normW, (np.linalg.norm(got - expect), normW)
    a = w["alpha0"]
    F64 = plan.rhs(_dev(a)).cpu().numpy()
    Nn = -(F64 + c["nu"] * lam * a)
    s = np.where(ms == 0, 1.0, 2.0)
    e = np.sum(s * np.conj(a) * Nn).real / (np.linalg.norm(a) * np.linalg.norm(Nn))
    z = np.sum(s * lam * np.conj(a) * Nn).real / (np.linalg.norm(lam * a) * np.linalg.norm(Nn))
    assert abs(e) < 1e-12 and abs(z) < 1e-12
    plan.set_precision("fp32")
    F32 = plan.rhs(_dev(a)).cpu().numpy()
    assert _rel(F32, F64) <= 3e-5


def test_plan_argument_errors():
    from paper_1009_3308_gb300 import Plan, SphnseError
    with pytest.raises(SphnseError, match="E_INEXACT"):
        Plan(31, 46, 92, 1e-2, 1.0)
    with pytest.raises(SphnseError, match="E_ARG"):
        Plan(31, 40, 96, 1e-2, 1.0)
    with pytest.raises(SphnseError, match="E_UNSUPPORTED"):
        Plan(31, 49, 98, 1e-2, 1.0)
    plan = _plan(7, 24, 1e-2, 1.0)
    with pytest.raises(ValueError):
        plan.rhs(torch.zeros(5, dtype=torch.complex128, device="cuda"))


def test_rhs_host_pipelined_matches_device_rhs():
    """sphnse_rhs_host: five pipelined calls with different host inputs (two
    staging slots reused) give exactly the device-buffer RHS of each input."""
    from paper_1009_3308_gb300 import Plan
    L, nlon = 63, 192
    plan = Plan(L, nlon // 2, nlon, 1e-3, 1.0, precision="fp32")
    ins = [torch.from_numpy(coefficients(L, 70 + i, 0.05)).pin_memory() for i in range(5)]
    f = torch.from_numpy(coefficients(L, 80, 0.3)).pin_memory()
    outs = [torch.empty_like(x).pin_memory() for x in ins]
    tks = [plan.rhs_host(x, o, forcing_h=f) for x, o in zip(ins, outs)]
    plan.host_wait(tks[-1])
    for x, o in zip(ins, outs):
        ref = plan.rhs(x.cuda(), forcing=f.cuda()).cpu()
        assert torch.equal(o, ref)


@pytest.mark.parametrize("L,nlon", [(127, 384), (511, 1536)])
def test_rhs_host_direct_output_matches_device_rhs(L, nlon):
    """On the fused tensor-core RHS with a page-locked output array, the
    analysis writes F straight into it and reports completion in a mapped
    host flag: six calls with different inputs, with and without a forcing,
    mixing page-locked and pageable outputs (direct and copy-back calls share
    the staging slots), waited out of order, give exactly the device-buffer
    RHS of each input."""
    from paper_1009_3308_gb300 import Plan
    plan = Plan(L, nlon // 2, nlon, 1e-4, 1.0, precision="bf16x3")
    ins = [torch.from_numpy(coefficients(L, 90 + i, 0.02) * 3.0).pin_memory() for i in range(6)]
    f = torch.from_numpy(coefficients(L, 99, 0.3)).pin_memory()
    outs = [torch.empty_like(x) if i in (2, 3) else torch.empty_like(x).pin_memory() for i, x in enumerate(ins)]
    forc = [f if i % 2 else None for i in range(6)]
    tks = [plan.rhs_host(x, o, forcing_h=fo) for x, o, fo in zip(ins, outs, forc)]
    for i in (2, 5, 0, 4, 1, 3):
        plan.host_wait(tks[i])
    for x, o, fo in zip(ins, outs, forc):
        ref = plan.rhs(x.cuda(), forcing=None if fo is None else fo.cuda()).cpu()
        assert torch.equal(o, ref)
    assert plan.sync() == 0
