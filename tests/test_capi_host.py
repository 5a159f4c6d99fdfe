"""CPU checks of the C-ABI library: it loads, exports every entry point the
header declares, and its host FP64 precompute (Gauss nodes of Eq. (quadrule),
Legendre tables of Eq. (sph_har)) agrees with the oracle's independent one."""
import ctypes

import numpy as np
import pytest

from oracle.legendre import pt_table
from oracle.quadrature import gauss_legendre
from paper_1009_3308_gb300 import _capi


def _p(a):
    return a.ctypes.data_as(_capi.c_double_p)


def test_library_exports_every_declared_symbol():
    lib = _capi.lib()
    names = _capi.header_symbols()
    assert len(names) >= 15
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    assert set(names) <= set(_capi._SIGS), set(names) - set(_capi._SIGS)


@pytest.mark.parametrize("n", [1, 7, 48, 384, 768])
def test_host_gauss_nodes_match_oracle(n):
    lib = _capi.lib()
    th, x, s, w = (np.zeros(n) for _ in range(4))
    assert lib.sphnse_host_gauss_nodes(n, _p(th), _p(x), _p(s), _p(w)) == 0
    oth, ox, os_, ow = gauss_legendre(n)
    np.testing.assert_allclose(th, oth, rtol=4e-16, atol=0)
    np.testing.assert_allclose(x, ox, rtol=0, atol=4.5e-16)  # two ulps
    np.testing.assert_allclose(s, os_, rtol=4e-16)
    np.testing.assert_allclose(w, ow, rtol=2e-14)  # n eps of the recurrence


@pytest.mark.parametrize("Kmax,m", [(40, 0), (40, 17), (512, 0), (512, 300), (512, 511)])
def test_host_legendre_matches_oracle(Kmax, m):
    lib = _capi.lib()
    oth, ox, os_, _ = gauss_legendre(96)
    out = np.zeros((Kmax - m + 1) * ox.size)
    assert lib.sphnse_host_legendre(Kmax, m, ox.size, _p(ox), _p(os_), _p(out)) == 0
    got = out.reshape(Kmax - m + 1, ox.size)
    ref = pt_table(Kmax, ox, os_)[m] if Kmax <= 64 else None
    if ref is None:
        # only order m of the oracle table is needed: build it for Kmax on the fly
        ref = pt_table(Kmax, ox, os_)[m]
    scale = np.maximum(np.abs(ref), 1e-290)
    assert np.max(np.abs(got - ref) / scale * (np.abs(ref) > 1e-290)) < 1e-12
    assert np.all(np.abs(got[np.abs(ref) <= 1e-290]) < 1e-280)


def test_argument_errors_need_no_gpu():
    lib = _capi.lib()
    assert lib.sphnse_host_gauss_nodes(0, None, None, None, None) == -1
    assert lib.sphnse_host_legendre(3, 5, 4, None, None, None) == -1
    assert lib.sphnse_error_string(-2).decode().startswith("nlon < 3L+2")
