"""The four-step longitude transform (nlon = 24 M2) in its two CTA shapes:
128 threads per 128 / M2 rings, each thread carrying both packed spectra,
and 256 threads, one spectrum per thread (SPHNSE_KEY_RING_THREADS).  Every
spectrum sees the same FP32 operations in the same order, so the RHS must
agree bit for bit; oracle parity of the default shape is covered by the RHS
parity tests."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from seeded_inputs import coefficients

pytestmark = pytest.mark.gpu


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.complex128)).cuda()


@pytest.mark.parametrize("prec", ["fp32", "bf16x3"])
@pytest.mark.parametrize("L,nlat,nlon", [(127, 192, 384), (255, 384, 768), (511, 768, 1536)])
def test_ring_shapes_give_identical_rhs(L, nlat, nlon, prec):
    from paper_1009_3308_gb300 import Plan
    plan = Plan(L, nlat, nlon, 1e-4, 1.0, precision=prec)
    a = _dev(coefficients(L, 700 + L, 0.02) * 3.0)
    out = {}
    for nt in (128, 256, 0):
        plan.set("RING_THREADS", nt)
        assert plan.get("RING_THREADS") == nt
        out[nt] = plan.rhs(a).clone()
    assert plan.sync() == 0
    assert bool(torch.isfinite(torch.view_as_real(out[0])).all())
    assert torch.equal(out[128], out[256])
    assert torch.equal(out[0], out[256])


def test_ring_threads_rejects_other_shapes():
    from paper_1009_3308_gb300 import Plan, SphnseError
    plan = Plan(31, 48, 96, 1e-2, 1.0, precision="fp32")
    for bad in (64, 512, -1):
        with pytest.raises(SphnseError, match="E_ARG"):
            plan.set("RING_THREADS", bad)
    # M2 = 4 has no 256-thread shape: the setting falls back to 128 threads
    plan.set("RING_THREADS", 256)
    a = _dev(coefficients(31, 731, 0.3))
    f256 = plan.rhs(a).clone()
    plan.set("RING_THREADS", 128)
    assert torch.equal(f256, plan.rhs(a))
