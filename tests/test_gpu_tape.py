"""The checkpointed trajectory tape behind the C ABI (sphnse_tape_*,
sphnse_adjoint_step, sphnse_adjoint_run), called through ctypes without the
autograd layer:

* the reverse sweep the tape drives (segments replayed from checkpoints in
  the library) gives the gradient of a reverse sweep over explicitly stored
  states (sphnse_adjoint_step_explicit) on the adjoint workload: L = 255,
  384 x 768, 200 steps, checkpoints every 20;
* the gradient of the first 20-step segment of that workload matches the
  oracle's tangent-linear directional derivatives (Sec. 4.2, frozen
  controller), in two directions, one of them moving nu;
* misuse is an argument error, not a wrong answer.
"""
import ctypes
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle.ndf import NDF
from oracle.rhs import Problem, rhs_separable
from oracle.tlm import ReplayTLM
from seeded_inputs import random_packed, workload

pytestmark = pytest.mark.gpu


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.complex128)).cuda()


def _rdot(a, b):
    return float(np.sum(a.real * b.real + a.imag * b.imag))


def _p(t):
    return ctypes.c_void_p(t.data_ptr())


def _workload_plan():
    from paper_1009_3308_gb300 import Plan
    w = workload("adjoint")
    c = w["config"]
    plan = Plan(c["L"], c["nlat"], c["nlon"], c["nu"], c["Omega"])
    plan.set("RTOL", c["rtol"])
    plan.set("ATOL", 1e-3 * c["rtol"] * float(np.max(np.abs(w["alpha0"]))))
    return w, c, plan


def _schedule(plan, a0, nsteps):
    from paper_1009_3308_gb300 import Integrator
    it = Integrator(plan, _dev(a0))
    sched = []
    for _ in range(nsteps):
        info = it.step()
        sched.append((info["h"], info["order"]))
    return sched, it.h0


def _tape_gradient(plan, a0, sched, h0, checkpoint, lam_of_state):
    """Forward through a tape, then the library's reverse sweep on lam."""
    from paper_1009_3308_gb300 import _capi
    from paper_1009_3308_gb300._capi import StepInfo, check
    lib = _capi.lib()
    tape = ctypes.c_void_p()
    check("sphnse_tape_create", lib.sphnse_tape_create(plan.handle, len(sched), checkpoint, ctypes.byref(tape)))
    try:
        da0 = _dev(a0)
        plan._stream()
        check("sphnse_tape_begin", lib.sphnse_tape_begin(tape, _p(da0), 0.0, float(h0), None))
        info = StepInfo()
        for h, k in sched:
            check("sphnse_tape_record", lib.sphnse_tape_record(tape, float(h), int(k), 50, ctypes.byref(info)))
        aT = plan.empty_coeff()
        check("sphnse_tape_state", lib.sphnse_tape_state(tape, _p(aT)))
        lam = lam_of_state(aT)
        nub = ctypes.c_double(0.0)
        check("sphnse_adjoint_run", lib.sphnse_adjoint_run(plan.handle, tape, _p(lam), ctypes.byref(nub)))
        torch.cuda.synchronize()
        return aT.cpu().numpy(), lam.cpu().numpy(), nub.value
    finally:
        lib.sphnse_tape_destroy(tape)


def _explicit_gradient(plan, a0, sched, h0, lam_of_state):
    """The same gradient with every forward state stored by the caller and
    one sphnse_adjoint_step_explicit per step."""
    from paper_1009_3308_gb300 import Integrator, MAXK, _capi
    from paper_1009_3308_gb300._capi import check
    lib = _capi.lib()
    it = Integrator(plan, _dev(a0), h0=h0)
    states, hdif = [], []
    for h, k in sched:
        hdif.append(it.replay_step(h, k)["h_dif_before"])
        states.append(it.alpha.clone())
    lam = lam_of_state(it.alpha)
    dbar = torch.zeros((MAXK + 2, plan.n_coeff), dtype=torch.complex128, device="cuda")
    nub = ctypes.c_double(0.0)
    plan._stream()
    for i in range(len(sched) - 1, -1, -1):
        h, k = sched[i]
        check("sphnse_adjoint_step_explicit", lib.sphnse_adjoint_step_explicit(
            plan.handle, float(h), int(k), float(hdif[i]), _p(states[i]), _p(lam), _p(dbar), ctypes.byref(nub)))
    a0d = _dev(a0)
    check("sphnse_adjoint_init", lib.sphnse_adjoint_init(plan.handle, float(h0), _p(a0d), _p(lam), _p(dbar[0]),
                                                         ctypes.byref(nub)))
    torch.cuda.synchronize()
    return it.alpha.cpu().numpy(), lam.cpu().numpy(), nub.value


def test_tape_reverse_sweep_equals_explicit_states_L255_workload():
    w, c, plan = _workload_plan()
    a0 = w["alpha0"]
    tgt = _dev(w["target"])
    lo, hi = math.radians(30), math.radians(60)
    sched, h0 = _schedule(plan, a0, c["steps"])

    def grad_of(aT):
        return plan.objective(aT, tgt, lo, hi)[1]
    aT1, g1, n1 = _tape_gradient(plan, a0, sched, h0, c["checkpoint"], grad_of)
    aT2, g2, n2 = _explicit_gradient(plan, a0, sched, h0, grad_of)
    print(f"tape vs explicit: state {np.linalg.norm(aT1 - aT2) / np.linalg.norm(aT2):.2e}, "
          f"gradient {np.linalg.norm(g1 - g2) / np.linalg.norm(g2):.2e}, nu {abs(n1 - n2) / abs(n2):.2e}")
    assert np.linalg.norm(aT1 - aT2) <= 1e-14 * np.linalg.norm(aT2)
    assert np.linalg.norm(g1 - g2) <= 1e-12 * np.linalg.norm(g2)
    assert abs(n1 - n2) <= 1e-12 * abs(n2)


def test_adjoint_workload_gradient_matches_oracle_tlm():
    """First 20-step segment of the adjoint workload (L = 255), FP64: the
    tape gradient of w . alpha_20 with respect to alpha0 and nu against the
    oracle's tangent-linear model along two directions (dnu = 0 and
    dnu = 0.1 nu)."""
    w, c, plan = _workload_plan()
    a0 = w["alpha0"]
    nsteps = c["checkpoint"]
    sched, h0 = _schedule(plan, a0, nsteps)
    wv = random_packed(c["L"], 5501)
    _, g, gnu = _tape_gradient(plan, a0, sched, h0, c["checkpoint"], lambda aT: _dev(wv))
    prob = Problem(c["L"], c["nlon"], c["nu"], c["Omega"])
    jd = -prob.nu * prob.lam + 2j * prob.Omega * prob.ms / prob.lam
    for seed, dnu in ((5502, 0.0), (5503, 0.1 * c["nu"])):
        v = random_packed(c["L"], seed) * np.abs(a0).max()
        nd = NDF(lambda t, y: rhs_separable(prob, y), jd, 0.0, a0, rtol=c["rtol"], atol=1e-9, h0=h0)
        tl = ReplayTLM(prob, nd, v, dnu)
        for h, k in sched:
            tl.step(h, k)
        ref = _rdot(wv, tl.dy)
        got = _rdot(g, v) + gnu * dnu
        print(f"direction {seed}: adjoint {got:.15e} oracle TLM {ref:.15e} rel {abs(got - ref) / abs(ref):.2e}")
        assert abs(got - ref) <= 1e-9 * abs(ref), (seed, got, ref)


def test_tape_misuse_is_an_argument_error():
    from paper_1009_3308_gb300 import Plan, SphnseError, Tape
    plan = Plan(15, 24, 48, 1e-3, 1.0)
    a0 = _dev(random_packed(15, 3) * 0.1)
    tape = Tape(plan, 4, checkpoint_every=2)
    lam = _dev(random_packed(15, 4))
    with pytest.raises(SphnseError, match="E_ARG"):
        tape.adjoint_step(0, lam)                       # nothing recorded
    tape.begin(a0, h0=1e-3)
    for h, k in [(1e-3, 1), (1e-3, 2), (2e-3, 2), (2e-3, 3)]:
        tape.record(h, k)
    with pytest.raises(SphnseError, match="E_TOO_LARGE"):
        tape.record(2e-3, 3)                            # beyond max_steps
    with pytest.raises(SphnseError, match="E_ARG"):
        tape.adjoint_step(1, lam)                       # a sweep starts at the last step
    tape.adjoint_step(3, lam)
    with pytest.raises(SphnseError, match="E_ARG"):
        tape.adjoint_step(1, lam)                       # steps are taken in turn
    tape.adjoint_step(2, lam)
    plan.set("NU", 2e-3)
    with pytest.raises(SphnseError, match="E_ARG"):
        tape.adjoint_step(1, lam)                       # the map has changed
    plan.set("NU", 1e-3)
    tape.adjoint_step(1, lam)
    tape.adjoint_step(0, lam)
    assert tape.info()["nsteps"] == 4
    assert bool(torch.isfinite(torch.view_as_real(lam)).all())
