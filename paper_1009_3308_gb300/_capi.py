"""ctypes declarations of the libsphnse C ABI (include/sphnse.h).

Argument marshalling only: every entry point runs in the CUDA library.  If
the library is missing it is built in-tree (nvcc); if it cannot be built or
loaded, an ImportError is raised -- there is no other implementation.
"""
import ctypes
import os

from . import build as _build

c_double_p = ctypes.POINTER(ctypes.c_double)

SPHNSE_OK = 0
E_CODES = {-1: "E_ARG", -2: "E_INEXACT", -3: "E_NOMEM", -4: "E_CUDA", -5: "E_NONFINITE",
           -6: "E_STEP_TOO_SMALL", -7: "E_TIMEOUT", -8: "E_UNSUPPORTED", -9: "E_TOO_LARGE"}
KEY = dict(PRECISION=1, NU=2, OMEGA=3, RTOL=4, ATOL=5, MAX_ORDER=6, NEWTON_MAX_ITER=7,
           H_MAX=8, BDF=9, CORIOLIS_SPLIT=10, TIMING_PERIOD=11, N_COEFF=100, L=101, NLAT=102, NLON=103, TABLE_BYTES=104, ROUNDS=105,
           SYN_ENTRIES=106, ANA_ENTRIES=107, AUTOTUNE=12, BUCKETS=108, SYN_CLUSTER=14,
           RING_THREADS=13)
PRECISION = {"fp64": 0, "fp32": 1, "bf16x3": 2}
MAXK = 5
STAGES = ("prep", "synthesis", "ring", "analysis", "finish", "step", "transpose")


class State(ctypes.Structure):
    _fields_ = [("alpha", ctypes.c_void_p), ("dif", ctypes.c_void_p), ("t", ctypes.c_double),
                ("h", ctypes.c_double), ("t_end", ctypes.c_double), ("order", ctypes.c_int),
                ("nconhk", ctypes.c_int), ("havrate", ctypes.c_int), ("miter_k", ctypes.c_int),
                ("h_dif", ctypes.c_double), ("rate", ctypes.c_double), ("miter_h", ctypes.c_double)]


class StepInfo(ctypes.Structure):
    _fields_ = [("t", ctypes.c_double), ("h", ctypes.c_double), ("err", ctypes.c_double),
                ("order", ctypes.c_int), ("newton_iters", ctypes.c_int), ("rejections", ctypes.c_int),
                ("rhs_evals", ctypes.c_int), ("next_order", ctypes.c_int), ("next_h", ctypes.c_double),
                ("h_dif_before", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_SIGS = {
    "sphnse_plan_create": (ctypes.c_void_p, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double]),
    "sphnse_last_error": (ctypes.c_int, []),
    "sphnse_error_string": (ctypes.c_char_p, [ctypes.c_int]),
    "sphnse_plan_destroy": (None, [ctypes.c_void_p]),
    "sphnse_plan_set": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_double]),
    "sphnse_plan_get": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, c_double_p]),
    "sphnse_sync": (ctypes.c_int, [ctypes.c_void_p]),
    "sphnse_set_stream": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "sphnse_grid_nodes": (ctypes.c_int, [ctypes.c_void_p, c_double_p, c_double_p, c_double_p, c_double_p]),
    "sphnse_rhs": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_double, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "sphnse_grid_fields": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "sphnse_project": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "sphnse_state_init": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(State), ctypes.c_double, ctypes.c_double, ctypes.c_void_p]),
    "sphnse_step": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(State), ctypes.c_void_p, ctypes.POINTER(StepInfo)]),
    "sphnse_advance": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(State), ctypes.c_void_p, ctypes.c_int,
                                      ctypes.c_void_p]),
    "sphnse_replay_step": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(State), ctypes.c_void_p, ctypes.c_double,
                                          ctypes.c_int, ctypes.c_int, ctypes.POINTER(StepInfo)]),
    "sphnse_rhs_adjoint": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, c_double_p]),
    "sphnse_adjoint_step_explicit": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_double, ctypes.c_int, ctypes.c_double,
                                                    ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, c_double_p]),
    "sphnse_tape_create": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_void_p)]),
    "sphnse_tape_destroy": (None, [ctypes.c_void_p]),
    "sphnse_tape_begin": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_double, ctypes.c_double,
                                         ctypes.c_void_p]),
    "sphnse_tape_record": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_double, ctypes.c_int, ctypes.c_int,
                                          ctypes.POINTER(StepInfo)]),
    "sphnse_tape_info": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int), c_double_p, c_double_p]),
    "sphnse_tape_state": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "sphnse_adjoint_step": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p,
                                           c_double_p]),
    "sphnse_adjoint_run": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, c_double_p]),
    "sphnse_adjoint_init": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_double, ctypes.c_void_p, ctypes.c_void_p,
                                           ctypes.c_void_p, c_double_p]),
    "sphnse_objective": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_double,
                                        ctypes.c_double, c_double_p, ctypes.c_void_p]),
    "sphnse_ensemble_create": (ctypes.c_void_p, [ctypes.c_int, ctypes.POINTER(ctypes.c_int), c_double_p, ctypes.c_double]),
    "sphnse_ensemble_destroy": (None, [ctypes.c_void_p]),
    "sphnse_ensemble_set": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_double]),
    "sphnse_ensemble_get": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_double)]),
    "sphnse_ensemble_set_stream": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "sphnse_ensemble_bucket": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                               ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                               ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                               ctypes.POINTER(ctypes.c_double)]),
    "sphnse_ensemble_instance": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_void_p),
                                                ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_int)]),
    "sphnse_ensemble_rhs": (ctypes.c_int, [ctypes.c_void_p]),
    "sphnse_ensemble_init": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_double]),
    "sphnse_ensemble_step": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "sphnse_rhs_host": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_double, ctypes.c_void_p, ctypes.c_void_p,
                                       ctypes.c_void_p, ctypes.POINTER(ctypes.c_longlong)]),
    "sphnse_host_wait": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_longlong]),
    "sphnse_energy_spectrum": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "sphnse_resize": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]),
    "sphnse_inertial_manifold": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                                ctypes.c_void_p]),
    "sphnse_ensemble_advance": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]),
    "sphnse_stage_timing": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "sphnse_stage_times": (ctypes.c_int, [ctypes.c_void_p, c_double_p, ctypes.POINTER(ctypes.c_long)]),
    "sphnse_nu_sensitivity_noalloc": (ctypes.c_int, [ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                                      ctypes.c_void_p]),
    "sphnse_host_gauss_nodes": (ctypes.c_int, [ctypes.c_int, c_double_p, c_double_p, c_double_p, c_double_p]),
    "sphnse_host_legendre": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, c_double_p, c_double_p, c_double_p]),
}

_lib = None


def header_symbols():
    """Function names declared in include/sphnse.h."""
    import re
    hdr = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "sphnse.h")
    with open(hdr) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(sphnse_[a-z0-9_]+)\s*\(", text)))


def lib():
    """The loaded library (built on first use)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    try:
        if _build._stale():
            _build.build()
        L = ctypes.CDLL(path)
    except Exception as e:  # no silent fallback: the CUDA library is the implementation
        raise ImportError(f"libsphnse could not be built or loaded: {e}") from e
    for name, (res, args) in _SIGS.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


class SphnseError(RuntimeError):
    def __init__(self, fn, code):
        msg = lib().sphnse_error_string(code).decode()
        super().__init__(f"{fn} failed: {E_CODES.get(code, code)} ({msg})")
        self.code = code


def check(fn, code):
    if code < 0:
        raise SphnseError(fn, code)
    return code
