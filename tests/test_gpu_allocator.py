"""Library-owned device memory served by a caller's allocator
(nb_set_allocator): torch's caching allocator through the binding, and an
allocator that refuses every request."""
import ctypes
import gc

import pytest
import torch

from paper_1908_06091_b300 import nabla

pytestmark = pytest.mark.gpu

OPS = (("grad", 0, 2), ("div", 1, 1), ("curl", 1, 1), ("lap", 0, 1))


@pytest.fixture
def runtime_allocator_after():
    yield
    nabla.use_torch_allocator(False)


def _fields(meth, nlev, seed=3):
    fs = nabla.NodeColumns(meth, nlev, torch.float32)
    gen = torch.Generator(device="cuda").manual_seed(seed)
    f = fs.create_field()
    f.copy_(torch.randn(f.shape, device="cuda", generator=gen))
    uv = fs.create_field(nvar=2)
    uv.copy_(torch.randn(uv.shape, device="cuda", generator=gen))
    outs = {op: fs.create_field(nvar=nvar, fill=float("nan")) for op, _, nvar in OPS}
    return fs, (f, uv), outs


def _run_all(meth, ins, outs):
    for op, k, _ in OPS:
        nabla.apply(meth, op, ins[k], outs[op])  # Laplacian without scratch: library-owned buffer
    torch.cuda.synchronize()


def _settled():
    gc.collect()
    torch.cuda.synchronize()
    return torch.cuda.memory_allocated()


def test_torch_allocator_serves_method_plans_and_scratch(runtime_allocator_after):
    N, nlev = 64, 37
    meth_rt = nabla.Method(nabla.Mesh(nabla.Grid(N), 1))
    _, ins_rt, ref = _fields(meth_rt, nlev)
    _run_all(meth_rt, ins_rt, ref)
    mesh = nabla.Mesh(nabla.Grid(N), 1)
    base = _settled()
    nabla.use_torch_allocator(True)
    meth = nabla.Method(mesh)
    held = torch.cuda.memory_allocated() - base
    assert held >= meth.device_bytes() > 0
    fs, ins, got = _fields(meth, nlev)
    with_fields = _settled()
    _run_all(meth, ins, got)
    assert _settled() > with_fields  # the tile plans made on first use joined the method
    for op, _, _ in OPS:  # same kernels on the same data: bitwise equal
        assert torch.equal(got[op], ref[op]), op
    nabla.use_torch_allocator(False)
    del fs, ins, got, meth
    assert _settled() == base
    assert nabla.device_status() == 0


def test_torch_allocator_serves_batch_tables(runtime_allocator_after):
    meth = nabla.Method(nabla.Mesh(nabla.Grid(32), 1))
    fs, (f, _), outs = _fields(meth, 16, 5)
    lap_ref, lap = outs["lap"], outs["grad"][..., 0].contiguous()
    b_rt = nabla.Batch([("lap", meth, f, lap_ref)])
    b_rt.run()
    base = _settled()
    nabla.use_torch_allocator(True)
    b = nabla.Batch([("lap", meth, f, lap)])
    assert torch.cuda.memory_allocated() - base > 2 * lap.numel() * 4  # gradient scratch + tables
    b.run()
    torch.cuda.synchronize()
    assert torch.equal(lap, lap_ref)
    nabla.use_torch_allocator(False)
    del b
    assert _settled() == base
    assert nabla.device_status() == 0


def test_refusing_allocator_fails_cleanly_with_eoom(runtime_allocator_after):
    meth = nabla.Method(nabla.Mesh(nabla.Grid(16), 1))
    fs, (f, _), outs = _fields(meth, 8, 1)
    out = outs["lap"].fill_(0.0)
    calls = []

    def refuse(ctx, nbytes, stream):
        calls.append(nbytes)
        return None

    a = nabla.nb_allocator(None, nabla._ALLOC_FN(refuse), nabla._RELEASE_FN(lambda *args: None))
    L = nabla.lib()
    nabla.check(L.nb_set_allocator(ctypes.byref(a)))
    try:
        h = ctypes.c_void_p()
        assert L.nb_method_create(meth.mesh.handle, 0.0, ctypes.byref(h)) == nabla.NB_EOOM
        assert b"allocator callback returned NULL" in L.nb_last_error()
        before = nabla.launch_count()
        fi, fo = nabla.field_view(f, 1), nabla.field_view(out, 1)
        rc = L.nb_nabla_laplacian(meth.handle, ctypes.byref(fi), ctypes.byref(fo), None,
                                  ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
        assert rc == nabla.NB_EOOM
        assert nabla.launch_count() == before
        assert len(calls) == 2
    finally:
        nabla.check(L.nb_set_allocator(None))
    torch.cuda.synchronize()
    assert torch.count_nonzero(out).item() == 0
