"""Gradients of a final-time objective through the NDF time stepping
(discretise-then-differentiate, frozen controller), as a
``torch.autograd.Function``.

The differentiated map is the replay of a fixed step schedule
[(h_n, k_n)]: each step is ``sphnse_replay_step`` (predictor, corrector
iterated to convergence, difference update; Sec. 4.2, Eq. (ode_disc)) and its
reverse is ``sphnse_adjoint_step``, whose transposed corrector solve applies
J(alpha_{n+1})^T through the library's adjoint RHS.  The schedule is usually
recorded by an adaptive run (``adaptive_schedule``).  Forward states are
checkpointed every ``checkpoint`` steps and recomputed segment by segment in
the backward pass.

Inputs and outputs are real float64 views (``torch.view_as_real``) of the
packed complex coefficients; gradients are with respect to those real
components, and with respect to the viscosity nu.
"""
import ctypes
import math

import torch

from . import Integrator, _capi
from ._capi import MAXK, check


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def adaptive_schedule(plan, alpha0, nsteps, forcing=None, t0=0.0, h0=0.0):
    """Run ``nsteps`` adaptive steps; returns (alpha_T, schedule, h0) with
    schedule = [(h, k), ...] of the accepted steps."""
    integ = Integrator(plan, alpha0, t0=t0, h0=h0, forcing=forcing)
    sched = []
    for _ in range(nsteps):
        info = integ.step()
        sched.append((info["h"], info["order"]))
    return integ.alpha, sched, integ.h0


class _State:
    """Plain holder of (alpha, dif, controller scalars) for replay."""

    def __init__(self, plan, alpha, dif, st):
        self.alpha = alpha
        self.dif = dif
        self.st = _capi.State()
        ctypes.memmove(ctypes.addressof(self.st), ctypes.addressof(st), ctypes.sizeof(st))
        self.st.alpha = alpha.data_ptr()
        self.st.dif = dif.data_ptr()


def _init_state(plan, alpha0, h0, forcing):
    alpha = alpha0.clone()
    dif = torch.zeros((MAXK + 2, plan.n_coeff), dtype=torch.complex128, device=plan.device)
    st = _capi.State()
    st.alpha = alpha.data_ptr()
    st.dif = dif.data_ptr()
    st.t_end = math.inf
    plan._stream()
    check("sphnse_state_init", _capi.lib().sphnse_state_init(
        plan.handle, ctypes.byref(st), 0.0, float(h0), _ptr(forcing) if forcing is not None else None))
    return _State(plan, alpha, dif, st)


def _replay(plan, S, h, k, forcing, newton_max):
    info = _capi.StepInfo()
    check("sphnse_replay_step", _capi.lib().sphnse_replay_step(
        plan.handle, ctypes.byref(S.st), _ptr(forcing) if forcing is not None else None,
        float(h), int(k), int(newton_max), ctypes.byref(info)))
    return info.h_dif_before


def _snapshot(S):
    return (S.alpha.clone(), S.dif.clone(), S.st.h_dif, S.st.t)


def _restore(plan, snap, template_st):
    alpha, dif, h_dif, t = snap
    S = _State(plan, alpha.clone(), dif.clone(), template_st)
    S.st.h_dif = h_dif
    S.st.t = t
    return S


class _Trajectory(torch.autograd.Function):
    @staticmethod
    def forward(ctx, a0_real, nu, plan, schedule, h0, checkpoint, forcing, newton_max):
        plan.set("NU", float(nu))
        plan._stream()
        a0 = torch.view_as_complex(a0_real.contiguous()).clone()
        S = _init_state(plan, a0, h0, forcing)
        snaps = []
        hdif = []
        for i, (h, k) in enumerate(schedule):
            if i % checkpoint == 0:
                snaps.append(_snapshot(S))
            hdif.append(_replay(plan, S, h, k, forcing, newton_max))
        ctx.plan, ctx.schedule, ctx.h0 = plan, schedule, h0
        ctx.checkpoint, ctx.forcing, ctx.newton_max = checkpoint, forcing, newton_max
        ctx.snaps, ctx.hdif, ctx.a0, ctx.st = snaps, hdif, a0, S.st
        ctx.nu = float(nu)
        return torch.view_as_real(S.alpha.clone())

    @staticmethod
    def backward(ctx, gout):
        plan = ctx.plan
        plan.set("NU", ctx.nu)
        plan._stream()
        lib = _capi.lib()
        n = plan.n_coeff
        abar = torch.view_as_complex(gout.contiguous()).clone()
        dbar = torch.zeros((MAXK + 2, n), dtype=torch.complex128, device=plan.device)
        nub = ctypes.c_double(0.0)
        sched = ctx.schedule
        C = ctx.checkpoint
        nseg = len(ctx.snaps)
        for sgi in range(nseg - 1, -1, -1):
            lo, hi = sgi * C, min((sgi + 1) * C, len(sched))
            S = _restore(plan, ctx.snaps[sgi], ctx.st)
            states = []
            for i in range(lo, hi):
                h, k = sched[i]
                _replay(plan, S, h, k, ctx.forcing, ctx.newton_max)
                states.append(S.alpha.clone())
            for i in range(hi - 1, lo - 1, -1):
                h, k = sched[i]
                check("sphnse_adjoint_step", lib.sphnse_adjoint_step(
                    plan.handle, float(h), int(k), float(ctx.hdif[i]), _ptr(states[i - lo]),
                    _ptr(abar), _ptr(dbar), ctypes.byref(nub)))
        check("sphnse_adjoint_init", lib.sphnse_adjoint_init(
            plan.handle, float(ctx.h0), _ptr(ctx.a0), _ptr(abar), _ptr(dbar[0]), ctypes.byref(nub)))
        gnu = torch.tensor(nub.value, dtype=torch.float64)
        return torch.view_as_real(abar), gnu, None, None, None, None, None, None


def trajectory(plan, alpha0_real, nu, schedule, h0, checkpoint=20, forcing=None, newton_max=50):
    """alpha_T (real view) after replaying ``schedule`` from alpha0; differentiable
    with respect to ``alpha0_real`` and ``nu`` (0-d float64 tensor)."""
    return _Trajectory.apply(alpha0_real, nu, plan, list(schedule), float(h0), int(checkpoint), forcing,
                             int(newton_max))


class _Objective(torch.autograd.Function):
    @staticmethod
    def forward(ctx, a_real, plan, target, theta_lo, theta_hi):
        a = torch.view_as_complex(a_real.contiguous())
        J, grad = plan.objective(a, target, theta_lo, theta_hi)
        ctx.save_for_backward(torch.view_as_real(grad))
        return torch.tensor(J, dtype=torch.float64, device=a_real.device)

    @staticmethod
    def backward(ctx, gJ):
        (g,) = ctx.saved_tensors
        return g * gJ, None, None, None, None


def objective(plan, alpha_real, target, theta_lo, theta_hi):
    """Band kinetic energy + coefficient misfit (sphnse_objective), differentiable."""
    return _Objective.apply(alpha_real, plan, target, float(theta_lo), float(theta_hi))
