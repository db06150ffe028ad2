"""The allocation-free Laplacian (nb_nabla_laplacian_noalloc) against the
regular entry point nb_nabla_laplacian, both called through the C ABI.

This entry point exists for callers that cannot allocate device memory
while they run (a component with a device-memory budget fixed at start-up,
or a loop where cudaMalloc/cudaFree must not synchronise the device): its
intermediate gradient lives in a fixed scratch array inside the library.
The file is named to be collected last, so that a run stopping at the first
failure has already run every other test; it also passes on its own in a
fresh process."""
import ctypes

import numpy as np
import pytest
import torch

from paper_1908_06091_b300 import nabla

pytestmark = pytest.mark.gpu

TOL = {torch.float32: 1e-5, torch.float64: 1e-12}


def _lap_regular(meth, f, out):
    fi, fo = nabla.field_view(f, 1), nabla.field_view(out, 1)
    nabla.check(nabla.lib().nb_nabla_laplacian(meth.handle, ctypes.byref(fi), ctypes.byref(fo), None,
                                               ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)))


def _lap_noalloc(meth, f, out):
    fi, fo = nabla.field_view(f, 1), nabla.field_view(out, 1)
    return nabla.lib().nb_nabla_laplacian_noalloc(
        meth.handle, ctypes.byref(fi), ctypes.byref(fo),
        ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


def _rel(a, b):
    a, b = a.double(), b.double()
    return (torch.linalg.vector_norm(a - b) / torch.linalg.vector_norm(b)).item()


class _CountingAllocator:
    """A caller's allocator (nb_set_allocator) that counts the library's
    device allocations and serves them from torch's caching allocator."""

    def __init__(self):
        self.allocs = 0

        def alloc(ctx, nbytes, stream):
            self.allocs += 1
            return torch.cuda.caching_allocator_alloc(int(nbytes), stream=int(stream or 0))

        def release(ctx, ptr, nbytes, stream):
            torch.cuda.caching_allocator_delete(ptr)
        self._a = nabla.nb_allocator(None, nabla._ALLOC_FN(alloc), nabla._RELEASE_FN(release))

    def __enter__(self):
        nabla.check(nabla.lib().nb_set_allocator(ctypes.byref(self._a)))
        return self

    def __exit__(self, *exc):
        nabla.check(nabla.lib().nb_set_allocator(None))


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64], ids=["f32", "f64"])
def test_noalloc_laplacian_matches_regular_entry_twice_in_a_row(dtype):
    N, nlev = 48, 37
    meth = nabla.Method(nabla.Mesh(nabla.Grid(N), 1))
    fs = nabla.NodeColumns(meth, nlev, dtype)
    gen = torch.Generator(device="cuda").manual_seed(7)
    for call in range(2):  # second call: different input, scratch holds the first call's data
        f = fs.create_field()
        f.copy_(torch.randn(f.shape, dtype=dtype, device="cuda", generator=gen) * (1 + call))
        ref = fs.create_field(fill=float("nan"))
        got = fs.create_field(fill=float("nan"))
        with _CountingAllocator() as counter:
            _lap_regular(meth, f, ref)  # library scratch: one allocation through the caller's allocator
            torch.cuda.synchronize()
            assert counter.allocs >= 1
            counter.allocs = 0
            free0 = torch.cuda.mem_get_info()[0]
            assert _lap_noalloc(meth, f, got) == nabla.NB_OK, nabla.lib().nb_last_error()
            torch.cuda.synchronize()
            assert counter.allocs == 0
            if call == 1:  # the array was taken on the first call; nothing is allocated now
                assert torch.cuda.mem_get_info()[0] == free0
        assert torch.isfinite(got).all()
        assert _rel(got, ref) <= TOL[dtype], (call, _rel(got, ref))
    assert nabla.device_status() == 0


def test_noalloc_laplacian_rejects_problems_larger_than_its_scratch():
    # O200 x 137 levels in FP64 needs 167,200 x 138 x 2 x 8 bytes > 64 MiB
    meth = nabla.Method(nabla.Mesh(nabla.Grid(200), 1))
    fs = nabla.NodeColumns(meth, 137, torch.float64)
    f, out = fs.create_field(fill=1.0), fs.create_field(fill=0.0)
    need = meth.mesh.V * 138 * 2 * 8
    assert need > nabla.NOALLOC_SCRATCH_BYTES
    before = nabla.launch_count()
    rc = _lap_noalloc(meth, f, out)
    assert rc == nabla.NB_ESHAPE
    assert b"scratch" in nabla.lib().nb_last_error()
    assert nabla.launch_count() == before
    torch.cuda.synchronize()
    assert torch.count_nonzero(out).item() == 0
