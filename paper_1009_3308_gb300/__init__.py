"""GB300-native pseudospectral quadrature method for the Navier-Stokes
equations on the rotating unit sphere (Ganesh, Le Gia & Sloan).

Thin Python layer over the C ABI of ``libsphnse`` (include/sphnse.h):
argument marshalling of PyTorch CUDA tensors and streams only.  Every step of
the computation runs in the library's CUDA kernels; there is no CPU path.

Coefficient vectors are complex128 CUDA tensors in the packed order
(m = 0..L, then degree max(m,1)..L); grid arrays are float64 [nlat, nlon].
"""
import ctypes
import math

from . import _capi
from ._capi import KEY, MAXK, PRECISION, SphnseError, State, StepInfo, check

__all__ = ["Plan", "Integrator", "Tape", "Ensemble", "SphnseError", "PRECISION", "MAXK", "n_coeff"]


def n_coeff(L):
    return (L + 1) * (L + 2) // 2 - 1


def _torch():
    import torch
    return torch


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


class Plan:
    """One truncation degree L on the nlat x nlon Gauss-rectangle grid."""

    def __init__(self, L, nlat, nlon, nu, Omega, precision="fp64", device=None):
        torch = _torch()
        if not torch.cuda.is_available():
            raise RuntimeError("libsphnse runs on a CUDA device; none is available")
        self.device = torch.device(device if device is not None else "cuda")
        lib = _capi.lib()
        with torch.cuda.device(self.device):
            h = lib.sphnse_plan_create(int(L), int(nlat), int(nlon), float(nu), float(Omega))
        if not h:
            raise SphnseError("sphnse_plan_create", lib.sphnse_last_error())
        self._h = ctypes.c_void_p(h)
        self.L, self.nlat, self.nlon = int(L), int(nlat), int(nlon)
        self.n_coeff = n_coeff(L)
        self.set_precision(precision)

    # -- lifecycle -------------------------------------------------------
    def close(self):
        if getattr(self, "_h", None):
            _capi.lib().sphnse_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- parameters -------------------------------------------------------
    def set(self, key, value):
        check("sphnse_plan_set", _capi.lib().sphnse_plan_set(self._h, KEY[key], float(value)))

    def get(self, key):
        v = ctypes.c_double()
        check("sphnse_plan_get", _capi.lib().sphnse_plan_get(self._h, KEY[key], ctypes.byref(v)))
        return v.value

    def set_precision(self, precision):
        self.set("PRECISION", PRECISION[precision])
        self.precision = precision

    def sync(self):
        """Wait for the plan's stream; raises on a device-side timeout."""
        return check("sphnse_sync", _capi.lib().sphnse_sync(self._h))

    @property
    def handle(self):
        return self._h

    def nodes(self):
        """(theta, x, sin_theta, w) as float64 CPU tensors."""
        torch = _torch()
        arrs = [torch.empty(self.nlat, dtype=torch.float64) for _ in range(4)]
        ptrs = [ctypes.cast(a.data_ptr(), _capi.c_double_p) for a in arrs]
        check("sphnse_grid_nodes", _capi.lib().sphnse_grid_nodes(self._h, *ptrs))
        return tuple(arrs)

    def _stream(self):
        torch = _torch()
        s = torch.cuda.current_stream(self.device).cuda_stream
        check("sphnse_set_stream", _capi.lib().sphnse_set_stream(self._h, ctypes.c_void_p(s)))

    def _coeff(self, a, name):
        torch = _torch()
        if a is None:
            return None
        if a.dtype != torch.complex128 or not a.is_cuda or not a.is_contiguous() or a.numel() != self.n_coeff:
            raise ValueError(f"{name} must be a contiguous complex128 CUDA tensor of {self.n_coeff} entries")
        return a

    def empty_coeff(self):
        torch = _torch()
        return torch.empty(self.n_coeff, dtype=torch.complex128, device=self.device)

    # -- hot path ---------------------------------------------------------
    def rhs(self, alpha, forcing=None, out=None, t=0.0):
        """F(t, alpha) of Eq. (ode)."""
        alpha = self._coeff(alpha, "alpha")
        forcing = self._coeff(forcing, "forcing")
        out = self.empty_coeff() if out is None else self._coeff(out, "out")
        self._stream()
        check("sphnse_rhs", _capi.lib().sphnse_rhs(self._h, float(t), _ptr(alpha), _ptr(forcing), _ptr(out)))
        return out

    def rhs_host(self, alpha_h, out_h, forcing_h=None, t=0.0):
        """Pipelined F(alpha) from host tensors (complex128, pinned for
        overlap): returns a ticket; out_h is valid after host_wait(ticket).
        The arrays must stay alive and alpha_h / forcing_h unmodified until then."""
        torch = _torch()
        for name, a in (("alpha_h", alpha_h), ("out_h", out_h), ("forcing_h", forcing_h)):
            if a is None:
                continue
            if a.dtype != torch.complex128 or a.is_cuda or not a.is_contiguous() or a.numel() != self.n_coeff:
                raise ValueError(f"{name} must be a contiguous complex128 host tensor of {self.n_coeff} entries")
        tk = ctypes.c_longlong()
        self._stream()
        check("sphnse_rhs_host", _capi.lib().sphnse_rhs_host(self._h, float(t), _ptr(alpha_h), _ptr(forcing_h),
                                                             _ptr(out_h), ctypes.byref(tk)))
        return tk.value

    def host_wait(self, ticket):
        check("sphnse_host_wait", _capi.lib().sphnse_host_wait(self._h, int(ticket)))

    def grid_fields(self, alpha):
        """(zeta, u_theta, u_phi) on the grid, float64 [nlat, nlon] CUDA tensors."""
        torch = _torch()
        alpha = self._coeff(alpha, "alpha")
        outs = [torch.empty(self.nlat, self.nlon, dtype=torch.float64, device=self.device) for _ in range(3)]
        self._stream()
        check("sphnse_grid_fields", _capi.lib().sphnse_grid_fields(self._h, _ptr(alpha), *[_ptr(o) for o in outs]))
        return tuple(outs)

    def project(self, v_theta, v_phi, out=None):
        """(v, Z_{L,m})_M for a tangential grid field."""
        out = self.empty_coeff() if out is None else self._coeff(out, "out")
        for v in (v_theta, v_phi):
            if v.dtype != _torch().float64 or not v.is_contiguous() or v.shape != (self.nlat, self.nlon):
                raise ValueError("grid fields must be contiguous float64 [nlat, nlon]")
        self._stream()
        check("sphnse_project", _capi.lib().sphnse_project(self._h, _ptr(v_theta), _ptr(v_phi), _ptr(out)))
        return out

    # -- diagnostics (Sec. 6.2) -------------------------------------------
    def energy_spectrum(self, alpha):
        """E(L), L = 0..L_plan, of Eq. (energy): float64 CUDA tensor."""
        torch = _torch()
        alpha = self._coeff(alpha, "alpha")
        E = torch.empty(self.L + 1, dtype=torch.float64, device=self.device)
        self._stream()
        check("sphnse_energy_spectrum", _capi.lib().sphnse_energy_spectrum(self._h, _ptr(alpha), _ptr(E)))
        return E

    def resize(self, alpha_in, N_in, L_max=-1, out=None):
        """A field of truncation N_in in this plan's layout (modes above
        min(N_in, N, L_max) zero); L_max = N1 gives P_{N1}."""
        torch = _torch()
        if alpha_in.dtype != torch.complex128 or not alpha_in.is_cuda or not alpha_in.is_contiguous() \
                or alpha_in.numel() != (N_in + 1) * (N_in + 2) // 2 - 1:
            raise ValueError("alpha_in must be a packed complex128 CUDA tensor of truncation N_in")
        out = self.empty_coeff() if out is None else self._coeff(out, "out")
        self._stream()
        check("sphnse_resize", _capi.lib().sphnse_resize(self._h, int(N_in), _ptr(alpha_in), int(L_max), _ptr(out)))
        return out

    def inertial_manifold(self, N1, alpha, forcing=None, out=None):
        """Phi(P_{N1} alpha) of Eq. (eq:p-p) with N2 = this plan's N."""
        alpha = self._coeff(alpha, "alpha")
        forcing = self._coeff(forcing, "forcing")
        out = self.empty_coeff() if out is None else self._coeff(out, "out")
        self._stream()
        check("sphnse_inertial_manifold", _capi.lib().sphnse_inertial_manifold(
            self._h, int(N1), _ptr(alpha), _ptr(forcing), _ptr(out)))
        return out

    # -- adjoint ----------------------------------------------------------
    def rhs_adjoint(self, alpha, w, out=None, want_nu=False):
        """J(alpha)^T w (packed real components); with want_nu also <w, dF/dnu>."""
        alpha = self._coeff(alpha, "alpha")
        w = self._coeff(w, "w")
        out = self.empty_coeff() if out is None else self._coeff(out, "out")
        nb = ctypes.c_double(0.0)
        self._stream()
        check("sphnse_rhs_adjoint", _capi.lib().sphnse_rhs_adjoint(
            self._h, _ptr(alpha), _ptr(w), _ptr(out), ctypes.byref(nb) if want_nu else None))
        return (out, nb.value) if want_nu else out

    def objective(self, alpha, target, theta_lo, theta_hi):
        """(J, dJ/dalpha) of the band-energy + misfit objective."""
        alpha = self._coeff(alpha, "alpha")
        target = self._coeff(target, "target")
        grad = self.empty_coeff()
        J = ctypes.c_double()
        self._stream()
        check("sphnse_objective", _capi.lib().sphnse_objective(
            self._h, _ptr(alpha), _ptr(target), float(theta_lo), float(theta_hi), ctypes.byref(J), _ptr(grad)))
        return J.value, grad


class Integrator:
    """Adaptive NDF integrator state (sphnse_state) on a plan."""

    def __init__(self, plan, alpha0, t0=0.0, h0=0.0, forcing=None, t_end=math.inf):
        torch = _torch()
        self.plan = plan
        self.alpha = plan._coeff(alpha0, "alpha0").clone()
        self.dif = torch.zeros((MAXK + 2, plan.n_coeff), dtype=torch.complex128, device=plan.device)
        self.forcing = plan._coeff(forcing, "forcing")
        self.st = State()
        self.st.alpha = self.alpha.data_ptr()
        self.st.dif = self.dif.data_ptr()
        self.st.t_end = float(t_end)
        plan._stream()
        check("sphnse_state_init", _capi.lib().sphnse_state_init(
            plan.handle, ctypes.byref(self.st), float(t0), float(h0), _ptr(self.forcing)))
        self.h0 = self.st.h

    @property
    def t(self):
        return self.st.t

    def step(self):
        info = StepInfo()
        self.plan._stream()
        check("sphnse_step", _capi.lib().sphnse_step(
            self.plan.handle, ctypes.byref(self.st), _ptr(self.forcing), ctypes.byref(info)))
        return info.as_dict()

    def advance(self, nsteps):
        """nsteps accepted steps in one library call; their infos."""
        infos = (StepInfo * int(nsteps))()
        self.plan._stream()
        check("sphnse_advance", _capi.lib().sphnse_advance(
            self.plan.handle, ctypes.byref(self.st), _ptr(self.forcing), int(nsteps), ctypes.cast(infos, ctypes.c_void_p)))
        return [x.as_dict() for x in infos]

    def replay_step(self, h, k, newton_max=50):
        info = StepInfo()
        self.plan._stream()
        check("sphnse_replay_step", _capi.lib().sphnse_replay_step(
            self.plan.handle, ctypes.byref(self.st), _ptr(self.forcing), float(h), int(k), int(newton_max),
            ctypes.byref(info)))
        return info.as_dict()


class Tape:
    """Checkpointed trajectory tape of a plan (sphnse_tape): records the replay
    of a step schedule and drives the reverse sweep in the library."""

    def __init__(self, plan, max_steps, checkpoint_every=20):
        h = ctypes.c_void_p()
        check("sphnse_tape_create", _capi.lib().sphnse_tape_create(plan.handle, int(max_steps),
                                                                   int(checkpoint_every), ctypes.byref(h)))
        self._h = h
        self.plan = plan
        self._forcing = None

    def close(self):
        if getattr(self, "_h", None):
            _capi.lib().sphnse_tape_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def begin(self, alpha0, t0=0.0, h0=0.0, forcing=None):
        """Start at (t0, alpha0); h0 <= 0 picks the initial step.  The forcing
        tensor is kept alive by the tape object until the next begin."""
        alpha0 = self.plan._coeff(alpha0, "alpha0")
        self._forcing = self.plan._coeff(forcing, "forcing")
        self.plan._stream()
        check("sphnse_tape_begin", _capi.lib().sphnse_tape_begin(self._h, _ptr(alpha0), float(t0), float(h0),
                                                                 _ptr(self._forcing)))

    def record(self, h, k, newton_max=50):
        info = StepInfo()
        self.plan._stream()
        check("sphnse_tape_record", _capi.lib().sphnse_tape_record(self._h, float(h), int(k), int(newton_max),
                                                                   ctypes.byref(info)))
        return info.as_dict()

    def info(self):
        n, t, h0 = ctypes.c_int(), ctypes.c_double(), ctypes.c_double()
        check("sphnse_tape_info", _capi.lib().sphnse_tape_info(self._h, ctypes.byref(n), ctypes.byref(t),
                                                               ctypes.byref(h0)))
        return dict(nsteps=n.value, t=t.value, h0=h0.value)

    def state(self, out=None):
        out = self.plan.empty_coeff() if out is None else self.plan._coeff(out, "out")
        self.plan._stream()
        check("sphnse_tape_state", _capi.lib().sphnse_tape_state(self._h, _ptr(out)))
        return out

    def adjoint_step(self, step_index, lam):
        """Reverse of recorded step step_index on lam (in place); returns its dJ/dnu part."""
        lam = self.plan._coeff(lam, "lambda")
        nb = ctypes.c_double(0.0)
        self.plan._stream()
        check("sphnse_adjoint_step", _capi.lib().sphnse_adjoint_step(
            self.plan.handle, self._h, int(step_index), _ptr(lam), ctypes.byref(nb)))
        return nb.value

    def adjoint_run(self, lam):
        """The whole reverse sweep on lam (in place: dJ/dalpha(t_n) in,
        dJ/dalpha0 out); returns dJ/dnu."""
        lam = self.plan._coeff(lam, "lambda")
        nb = ctypes.c_double(0.0)
        self.plan._stream()
        check("sphnse_adjoint_run", _capi.lib().sphnse_adjoint_run(self.plan.handle, self._h, _ptr(lam),
                                                                   ctypes.byref(nb)))
        return nb.value


class Ensemble:
    """Batched ensemble of independent problems (sphnse_ensemble)."""

    def __init__(self, Ls, nus, Omega, device=None, precision="fp32", autotune=True, cluster=1):
        torch = _torch()
        if not torch.cuda.is_available():
            raise RuntimeError("libsphnse runs on a CUDA device; none is available")
        self.device = torch.device(device if device is not None else "cuda")
        lib = _capi.lib()
        n = len(Ls)
        Larr = (ctypes.c_int * n)(*[int(x) for x in Ls])
        narr = (ctypes.c_double * n)(*[float(x) for x in nus])
        with torch.cuda.device(self.device):
            h = lib.sphnse_ensemble_create(n, Larr, narr, float(Omega))
        if not h:
            raise SphnseError("sphnse_ensemble_create", -1)
        self._h = ctypes.c_void_p(h)
        self.n = n
        self.Ls = list(Ls)
        self.set("AUTOTUNE", 1 if autotune else 0)
        self.set("SYN_CLUSTER", cluster)
        if precision != "fp32":
            self.set_precision(precision)

    def buckets(self):
        """Per truncation bucket: L, instances, and on the tensor-core path the
        synthesis shape (instances per group, pipeline stages, CTAs per
        cluster) with its tuned duration in microseconds."""
        out = []
        for b in range(int(self.get("BUCKETS"))):
            L, cnt, grp, st, cl = (ctypes.c_int() for _ in range(5))
            us = ctypes.c_double()
            check("sphnse_ensemble_bucket", _capi.lib().sphnse_ensemble_bucket(
                self._h, b, ctypes.byref(L), ctypes.byref(cnt), ctypes.byref(grp), ctypes.byref(st),
                ctypes.byref(cl), ctypes.byref(us)))
            out.append(dict(L=L.value, instances=cnt.value, group=grp.value, stages=st.value, cluster=cl.value,
                            syn_us=us.value))
        return out

    def set_precision(self, precision):
        """"fp32" (streaming FP32 contractions) or "bf16x3" (the instances of
        each truncation share every table tile of a tensor-core synthesis)."""
        self.set("PRECISION", PRECISION[precision])

    def close(self):
        if getattr(self, "_h", None):
            _capi.lib().sphnse_ensemble_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set(self, key, value):
        check("sphnse_ensemble_set", _capi.lib().sphnse_ensemble_set(self._h, KEY[key], float(value)))

    def get(self, key, i=None, field="alpha"):
        """get("KEY") reads an ensemble parameter (e.g. "ROUNDS"); get(i) /
        get(i, "F") a copy of instance i's state or last RHS."""
        if isinstance(key, str):
            v = ctypes.c_double()
            check("sphnse_ensemble_get", _capi.lib().sphnse_ensemble_get(self._h, KEY[key], ctypes.byref(v)))
            return v.value
        return self._get_instance(key, field if i is None else i)

    def _stream(self):
        torch = _torch()
        s = torch.cuda.current_stream(self.device).cuda_stream
        check("sphnse_ensemble_set_stream", _capi.lib().sphnse_ensemble_set_stream(self._h, ctypes.c_void_p(s)))

    def _ptrs(self, i):
        a, f, nc = ctypes.c_void_p(), ctypes.c_void_p(), ctypes.c_int()
        check("sphnse_ensemble_instance", _capi.lib().sphnse_ensemble_instance(
            self._h, int(i), ctypes.byref(a), ctypes.byref(f), ctypes.byref(nc)))
        return a.value, f.value, nc.value

    def set_alpha(self, i, alpha):
        """Copy a complex128 CUDA tensor into instance i's state."""
        torch = _torch()
        a, _, nc = self._ptrs(i)
        if alpha.numel() != nc:
            raise ValueError(f"instance {i} has {nc} coefficients")
        src = alpha.to(self.device, torch.complex128).contiguous()
        torch.cuda.current_stream(self.device).synchronize()
        _cudart_copy(a, src.data_ptr(), nc * 16)

    def _get_instance(self, i, which="alpha"):
        """Copy of instance i's state ('alpha') or last RHS ('F')."""
        torch = _torch()
        a, f, nc = self._ptrs(i)
        out = torch.empty(nc, dtype=torch.complex128, device=self.device)
        torch.cuda.current_stream(self.device).synchronize()
        _cudart_copy(out.data_ptr(), a if which == "alpha" else f, nc * 16)
        return out

    def rhs(self):
        self._stream()
        check("sphnse_ensemble_rhs", _capi.lib().sphnse_ensemble_rhs(self._h))

    def init(self, t0=0.0):
        self._stream()
        check("sphnse_ensemble_init", _capi.lib().sphnse_ensemble_init(self._h, float(t0)))

    def step(self):
        infos = (StepInfo * self.n)()
        self._stream()
        check("sphnse_ensemble_step", _capi.lib().sphnse_ensemble_step(self._h, ctypes.cast(infos, ctypes.c_void_p)))
        return [x.as_dict() for x in infos]

    def advance(self, nsteps):
        """nsteps accepted steps of every instance, each at its own pace
        (asynchronous rounds); per instance the info of its last step, with
        Newton iterations, RHS evaluations and rejections summed over the call."""
        infos = (StepInfo * self.n)()
        self._stream()
        check("sphnse_ensemble_advance", _capi.lib().sphnse_ensemble_advance(
            self._h, int(nsteps), ctypes.cast(infos, ctypes.c_void_p)))
        return [x.as_dict() for x in infos]


def _cudart_copy(dst, src, nbytes):
    """Device-to-device copy of raw device memory through torch."""
    torch = _torch()
    src_t = _wrap(src, nbytes)
    dst_t = _wrap(dst, nbytes)
    dst_t.copy_(src_t)
    torch.cuda.current_stream().synchronize()


def _wrap(ptr, nbytes):
    torch = _torch()
    # a uint8 CUDA tensor view of raw device memory (CUDA array interface)
    class _Holder:
        __cuda_array_interface__ = {"shape": (nbytes,), "typestr": "|u1", "data": (int(ptr), False), "version": 2}
    return torch.as_tensor(_Holder(), device="cuda")
