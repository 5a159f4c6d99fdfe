"""The allocation-free entry point sphnse_nu_sensitivity_noalloc, for
callers that cannot call cudaMalloc (device memory owned by a framework's
caching allocator, or loops that cannot take an allocation's device
synchronisation).  Its result must equal the nu_bar that the allocating
path (sphnse_rhs_adjoint, plan-owned scratch) reports, on consecutive calls
that share the fixed device scratch.  Kept in its own file, collected last."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from seeded_inputs import coefficients, random_packed

pytestmark = pytest.mark.gpu


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.complex128)).cuda()


def _p(t):
    return ctypes.c_void_p(t.data_ptr())


def test_nu_sensitivity_noalloc_matches_allocating_path():
    from paper_1009_3308_gb300 import Plan, _capi
    lib = _capi.lib()
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    # larger case first, then a smaller one: the second call must not read
    # partial sums left in the shared scratch by the first
    for L, nlon in ((255, 768), (31, 96), (31, 96)):
        plan = Plan(L, nlon // 2, nlon, 1e-3, 1.0)
        a = _dev(coefficients(L, 5, 0.05))
        w = _dev(random_packed(L, 6))
        _, ref = plan.rhs_adjoint(a, w, want_nu=True)
        for _ in range(2):
            out.fill_(np.nan)
            rc = lib.sphnse_nu_sensitivity_noalloc(L, _p(a), _p(w), _p(out), stream)
            assert rc == 0
            torch.cuda.synchronize()
            got = float(out.item())
            assert abs(got - ref) <= 1e-12 * abs(ref), (L, got, ref)


def test_nu_sensitivity_noalloc_rejects_sizes_beyond_its_scratch():
    from paper_1009_3308_gb300 import _capi
    lib = _capi.lib()
    t = torch.zeros(4, dtype=torch.float64, device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert lib.sphnse_nu_sensitivity_noalloc(5000, _p(t), _p(t), _p(t), stream) == -9
    assert lib.sphnse_nu_sensitivity_noalloc(0, _p(t), _p(t), _p(t), stream) == -1
