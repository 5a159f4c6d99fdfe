"""Gradients of a final-time objective through the NDF time stepping
(discretise-then-differentiate, frozen controller), as a
``torch.autograd.Function``.

The differentiated map is the replay of a fixed step schedule
[(h_n, k_n)]: each step is the library's replay step (predictor, corrector
iterated to convergence, difference update; Sec. 4.2, Eq. (ode_disc)).  The
schedule is usually recorded by an adaptive run (``adaptive_schedule``).
The checkpoint tape, the segment recomputation and the reverse steps all run
in the library (``sphnse_tape_*``, ``sphnse_adjoint_run``); this module only
hands tensors to them.

Inputs and outputs are real float64 views (``torch.view_as_real``) of the
packed complex coefficients; gradients are with respect to those real
components, and with respect to the viscosity nu.  The plan's viscosity is
set to nu for the library calls and restored afterwards.
"""
import torch

from . import Integrator, Tape


def adaptive_schedule(plan, alpha0, nsteps, forcing=None, t0=0.0, h0=0.0):
    """Run ``nsteps`` adaptive steps; returns (alpha_T, schedule, h0) with
    schedule = [(h, k), ...] of the accepted steps."""
    integ = Integrator(plan, alpha0, t0=t0, h0=h0, forcing=forcing)
    sched = []
    for _ in range(nsteps):
        info = integ.step()
        sched.append((info["h"], info["order"]))
    return integ.alpha, sched, integ.h0


class _NuSet:
    """Set the plan's viscosity for the duration of a block."""

    def __init__(self, plan, nu):
        self.plan, self.nu = plan, float(nu)

    def __enter__(self):
        self.prev = self.plan.get("NU")
        self.plan.set("NU", self.nu)

    def __exit__(self, *exc):
        self.plan.set("NU", self.prev)


class _Trajectory(torch.autograd.Function):
    @staticmethod
    def forward(ctx, a0_real, nu, plan, schedule, h0, checkpoint, forcing, newton_max):
        a0 = torch.view_as_complex(a0_real.contiguous())
        tape = Tape(plan, max(1, len(schedule)), checkpoint)
        with _NuSet(plan, float(nu)):
            tape.begin(a0, 0.0, h0, forcing)
            for h, k in schedule:
                tape.record(h, k, newton_max)
            aT = tape.state()
        ctx.plan, ctx.tape, ctx.nu = plan, tape, float(nu)
        ctx.nu_device, ctx.nu_dtype = nu.device, nu.dtype
        ctx.nsteps = len(schedule)
        return torch.view_as_real(aT)

    @staticmethod
    def backward(ctx, gout):
        lam = torch.view_as_complex(gout.contiguous()).clone()
        gnu = 0.0
        if ctx.nsteps:
            with _NuSet(ctx.plan, ctx.nu):
                gnu = ctx.tape.adjoint_run(lam)
        return (torch.view_as_real(lam), torch.tensor(gnu, dtype=ctx.nu_dtype, device=ctx.nu_device),
                None, None, None, None, None, None)


def trajectory(plan, alpha0_real, nu, schedule, h0, checkpoint=20, forcing=None, newton_max=50):
    """alpha_T (real view) after replaying ``schedule`` from alpha0; differentiable
    with respect to ``alpha0_real`` and ``nu`` (0-d float64 tensor)."""
    if not torch.is_tensor(nu):
        nu = torch.tensor(float(nu), dtype=torch.float64)
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
