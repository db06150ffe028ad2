"""NodeColumns reductions (nb_field_reduce) against numpy on the same data,
and the area-weighted norms against the dual volumes the mesh reports."""
import numpy as np
import pytest
import torch

from paper_1908_06091_b300 import nabla
from gpu_helpers import product

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64], ids=["f32", "f64"])
@pytest.mark.parametrize("nvar", [1, 2])
def test_reductions_match_numpy(dtype, nvar):
    g, m, meth = product(48)
    nlev = 7
    fs = nabla.NodeColumns(meth, nlev, dtype)
    x = fs.create_field(nvar=nvar, fill=float("nan"))  # padding stays NaN: must not be read
    gen = torch.Generator(device="cuda").manual_seed(3)
    x.copy_(torch.randn(x.shape, dtype=dtype, device="cuda", generator=gen) * 5 + 1)
    h = x.double().cpu().numpy().reshape(m.V, nlev, nvar)
    vol = meth.dual_volumes()
    ref = {"min": h.min(0), "max": h.max(0), "sum": h.sum(0),
           "area_mean": np.einsum("i,ilc->lc", vol, h) / vol.sum(),
           "area_rms": np.sqrt(np.einsum("i,ilc->lc", vol, h * h) / vol.sum())}
    for kind, r in ref.items():
        got = nabla.reduce(meth, x, kind, nvar)
        got = got.reshape(nlev, nvar)
        if kind in ("min", "max"):
            assert np.array_equal(got, r), kind
        else:
            assert np.allclose(got, r, rtol=1e-12, atol=1e-12 * np.abs(h).max() * (m.V if kind == "sum" else 1)), kind
        assert np.array_equal(got, nabla.reduce(meth, x, kind, nvar).reshape(nlev, nvar))  # deterministic


def test_area_mean_of_a_constant_and_bad_arguments():
    g, m, meth = product(32)
    fs = nabla.NodeColumns(meth, 3, torch.float64)
    x = fs.create_field(fill=2.5)
    assert np.allclose(nabla.reduce(meth, x, "area_mean"), 2.5, rtol=1e-14)
    assert np.allclose(nabla.reduce(meth, x, "area_rms"), 2.5, rtol=1e-14)
    import ctypes
    fv = nabla.field_view(x, 1)
    out = np.zeros(3)
    assert nabla.lib().nb_field_reduce(meth.handle, ctypes.byref(fv), 9, out.ctypes.data, None) == nabla.NB_EINVAL
    g2, m2, meth2 = product(16)
    assert nabla.lib().nb_field_reduce(meth2.handle, ctypes.byref(fv), 0, out.ctypes.data, None) == nabla.NB_ESHAPE
