"""Fused divergence + curl (nb_nabla_divcurl): each output equals the
single-operator pass bit for bit, and therefore meets the oracle gate; the
call checks d and z before any launch."""
import ctypes

import numpy as np
import pytest
import torch

from paper_1908_06091_b300 import nabla
from gpu_helpers import inputs, oracle_mesh, oracle_op, product, rel_l2, run_op, to_device, to_grid

pytestmark = pytest.mark.gpu

TOL = {torch.float64: 1e-12, torch.float32: 1e-5}


def _fused(meth, fs, uvd):
    d = fs.create_field(fill=float("nan"))
    z = fs.create_field(fill=float("nan"))
    nabla.divcurl(meth, uvd, d, z)
    torch.cuda.synchronize()
    assert nabla.device_status() == 0
    return d, z


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64], ids=["f32", "f64"])
@pytest.mark.parametrize("N,nlev", [(32, 137), (32, 7), (48, 37), (16, 16), (16, 21)])
def test_fused_outputs_equal_single_operator_passes(N, nlev, dtype):
    g, m, meth = product(N)
    om = oracle_mesh(N)
    _, uv = inputs(om, nlev, 10, dtype)
    fs = nabla.NodeColumns(meth, nlev, dtype)
    uvd = to_device(fs, uv, m.permutation(), 2)
    d, z = _fused(meth, fs, uvd)
    d1, z1 = run_op(meth, fs, "div", uvd), run_op(meth, fs, "curl", uvd)
    lv = slice(0, nlev)
    assert torch.equal(d[:, lv], d1[:, lv]) and torch.equal(z[:, lv], z1[:, lv])
    perm = m.permutation()
    for out, op in ((d, "div"), (z, "curl")):
        ref = oracle_op(om, op, uv.astype(np.float64))
        assert rel_l2(to_grid(out, perm), ref) <= TOL[dtype], op


def test_fused_o640_137_levels_meets_the_gate():
    N, nlev = 640, 137
    g, m, meth = product(N)
    om = oracle_mesh(N)
    _, uv = inputs(om, nlev, 40, torch.float32)
    fs = nabla.NodeColumns(meth, nlev, torch.float32)
    perm = m.permutation()
    d, z = _fused(meth, fs, to_device(fs, uv, perm, 2))
    for out, op in ((d, "div"), (z, "curl")):
        ref = oracle_op(om, op, uv.astype(np.float64))
        assert rel_l2(to_grid(out, perm), ref) <= TOL[torch.float32], op


def test_fused_call_checks_outputs_before_any_launch():
    g, m, meth = product(16)
    fs = nabla.NodeColumns(meth, 20, torch.float32)
    uv = fs.create_field(nvar=2, fill=1.0)
    d = fs.create_field(fill=0.0)
    L = nabla.lib()
    before = nabla.launch_count()
    fu, fd = nabla.field_view(uv, 2), nabla.field_view(d, 1)
    # z = d: outputs overlap
    assert L.nb_nabla_divcurl(meth.handle, ctypes.byref(fu), ctypes.byref(fd), ctypes.byref(fd),
                              None) == nabla.NB_ESHAPE
    # z with another node stride
    z = torch.zeros((m.V, 24), dtype=torch.float32, device="cuda")
    fz = nabla.field_view(z[:, :20], 1)
    assert L.nb_nabla_divcurl(meth.handle, ctypes.byref(fu), ctypes.byref(fd), ctypes.byref(fz),
                              None) == nabla.NB_ESHAPE
    assert nabla.launch_count() == before
    assert torch.count_nonzero(d).item() == 0


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64], ids=["f32", "f64"])
@pytest.mark.parametrize("nlev", [7, 137])
def test_gradlap_outputs_equal_gradient_and_laplacian_calls(nlev, dtype):
    """nb_nabla_gradlap: the Laplacian's divergence pass reads the gradient
    it returns; both outputs equal the single calls bit for bit."""
    g_, m, meth = product(32)
    om = oracle_mesh(32)
    f, _ = inputs(om, nlev, 10, dtype)
    fs = nabla.NodeColumns(meth, nlev, dtype)
    fd = to_device(fs, f, m.permutation(), 1)
    g = fs.create_field(nvar=2, fill=float("nan"))
    lap = fs.create_field(fill=float("nan"))
    nabla.gradlap(meth, fd, g, lap)
    torch.cuda.synchronize()
    lv = slice(0, nlev)
    assert torch.equal(g[:, lv], run_op(meth, fs, "grad", fd)[:, lv])
    assert torch.equal(lap[:, lv], run_op(meth, fs, "lap", fd)[:, lv])
    ref = oracle_op(om, "lap", f.astype(np.float64))
    assert rel_l2(to_grid(lap, m.permutation()), ref) <= TOL[dtype]
    # g may not alias the Laplacian output
    fl = nabla.field_view(lap, 1)
    fg = nabla.field_view(g, 2)
    fi = nabla.field_view(fd, 1)
    bad = nabla.nb_field.from_buffer_copy(fg)
    bad.data = fl.data
    assert nabla.lib().nb_nabla_gradlap(meth.handle, ctypes.byref(fi), ctypes.byref(bad), ctypes.byref(fl),
                                        None) != nabla.NB_OK


def test_operator_calls_capture_into_a_cuda_graph_after_first_use():
    """After one eager call (tile plans built), the staged operators, the
    fused calls and the Laplacian with library scratch (stream-ordered) can
    be captured in a CUDA graph; replays give the eager results bit for bit."""
    g_, m, meth = product(48)
    om = oracle_mesh(48)
    f, uv = inputs(om, 37, 10, torch.float32)
    perm = m.permutation()
    fs = nabla.NodeColumns(meth, 37, torch.float32)
    fd, uvd = to_device(fs, f, perm, 1), to_device(fs, uv, perm, 2)
    outs = [fs.create_field(nvar=2), fs.create_field(), fs.create_field(), fs.create_field(), fs.create_field()]
    s = torch.cuda.Stream()

    def step():
        nabla.gradlap(meth, fd, outs[0], outs[1], stream=s)
        nabla.divcurl(meth, uvd, outs[2], outs[3], stream=s)
        nabla.apply(meth, "lap", fd, outs[4], stream=s)

    with torch.cuda.stream(s):
        step()
    s.synchronize()
    eager = [o.clone() for o in outs]
    for o in outs:
        o.zero_()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=s):
        step()
    for _ in range(2):
        graph.replay()
    torch.cuda.synchronize()
    assert all(torch.equal(a, b) for a, b in zip(eager, outs))
    assert torch.equal(outs[1], outs[4])  # gradlap's Laplacian == nb_nabla_laplacian
    assert nabla.device_status() == 0


@pytest.mark.parametrize("N,nlev", [(32, 137), (48, 91), (24, 37), (16, 16)])
def test_item_shapes_give_identical_results(N, nlev):
    """The staged div / curl kernels give the same bits for every item shape
    (2 or 3 units per item, items per node rounded to a multiple of 8 or
    not): each level's arithmetic does not depend on the shape."""
    g, m, meth = product(N)
    om = oracle_mesh(N)
    _, uv = inputs(om, nlev, 10, torch.float32)
    fs = nabla.NodeColumns(meth, nlev, torch.float32)
    uvd = to_device(fs, uv, m.permutation(), 2)
    ref = None
    try:
        for units, aligned in ((2, 0), (2, 1), (3, 0), (3, 1), (0, -1)):
            meth.set_item_shape(units, aligned)
            d, z = _fused(meth, fs, uvd)
            d1 = run_op(meth, fs, "div", uvd)
            got = (d[:, :nlev].clone(), z[:, :nlev].clone(), d1[:, :nlev].clone())
            if ref is None:
                ref = got
            assert all(torch.equal(a, b) for a, b in zip(got, ref)), (units, aligned)
    finally:
        meth.set_item_shape(0, -1)
    with pytest.raises(nabla.NablaError):
        meth.set_item_shape(4, 0)


@pytest.mark.parametrize("N,nlev", [(32, 137), (48, 91), (24, 37), (16, 16)])
def test_node_pairs_give_identical_results(N, nlev):
    """Evaluating both nodes of a node pair in one consumer thread (the
    default) gives the same bits as evaluating every node alone, for the
    single div and curl passes and the fused pass and for each item shape:
    each node's terms are summed in its row order either way (mode 1: pairs
    in every pass, 0: none, -1: all but the fused pass)."""
    g, m, meth = product(N)
    assert (m.node_pairs() >= 0).mean() > 0.8
    om = oracle_mesh(N)
    _, uv = inputs(om, nlev, 11, torch.float32)
    fs = nabla.NodeColumns(meth, nlev, torch.float32)
    uvd = to_device(fs, uv, m.permutation(), 2)
    ref = None
    try:
        for pairs in (0, 1, -1):
            meth.set_node_pairs(pairs)
            for units, aligned in ((2, 0), (3, 1)):
                meth.set_item_shape(units, aligned)
                d, z = _fused(meth, fs, uvd)
                d1, z1 = run_op(meth, fs, "div", uvd), run_op(meth, fs, "curl", uvd)
                got = [t[:, :nlev].clone() for t in (d, z, d1, z1)]
                if ref is None:
                    ref = got
                assert all(torch.equal(a, b) for a, b in zip(got, ref)), (pairs, units, aligned)
    finally:
        meth.set_node_pairs(-1)
        meth.set_item_shape(0, -1)
    with pytest.raises(nabla.NablaError):
        lib = nabla.lib()
        nabla.check(lib.nb_method_set_node_pairs(meth.handle, 2))


@pytest.mark.parametrize("N,nlev", [(32, 137), (24, 37), (16, 16)])
def test_node_pairs_give_identical_gradients_and_laplacians(N, nlev):
    """The staged gradient (and the Laplacian built on it) gives the same
    bits with node pairs on and off."""
    g, m, meth = product(N)
    om = oracle_mesh(N)
    f, _ = inputs(om, nlev, 12, torch.float32)
    fs = nabla.NodeColumns(meth, nlev, torch.float32)
    fd = to_device(fs, f, m.permutation(), 1)
    got = {}
    try:
        for pairs in (0, 1):
            meth.set_node_pairs(pairs)
            got[pairs] = [run_op(meth, fs, op, fd)[:, :nlev].clone() for op in ("grad", "lap")]
    finally:
        meth.set_node_pairs(-1)
    assert all(torch.equal(a, b) for a, b in zip(got[0], got[1]))


@pytest.mark.parametrize("tile_nodes", [8, 13, 1024])
def test_node_pairs_across_tile_boundaries(tile_nodes):
    """Small tiles cut many node pairs, whose nodes then take single slots
    in their tiles; large tiles hold long slot lists.  Every staged pass
    still gives the same bits with pairs in every pass (1) and in none (0)."""
    N, nlev = 32, 37
    g, m, meth = product(N)
    om = oracle_mesh(N)
    f, uv = inputs(om, nlev, 13, torch.float32)
    fs = nabla.NodeColumns(meth, nlev, torch.float32)
    perm = m.permutation()
    fd, uvd = to_device(fs, f, perm, 1), to_device(fs, uv, perm, 2)
    got = {}
    try:
        meth.set_kernel(nabla.KERNEL_TILED, tile_nodes)
        for pairs in (0, 1):
            meth.set_node_pairs(pairs)
            d, z = _fused(meth, fs, uvd)
            outs = [run_op(meth, fs, "grad", fd), run_op(meth, fs, "div", uvd), run_op(meth, fs, "curl", uvd),
                    run_op(meth, fs, "lap", fd), d, z]
            got[pairs] = [o[:, :nlev].clone() for o in outs]
    finally:
        meth.set_kernel(nabla.KERNEL_AUTO, 0)
        meth.set_node_pairs(-1)
    assert all(torch.equal(a, b) for a, b in zip(got[0], got[1]))
    # and the paired results meet the oracle gate
    for out, op, x in ((got[1][0], "grad", f), (got[1][1], "div", uv), (got[1][3], "lap", f)):
        ref = oracle_op(om, op, x.astype(np.float64))
        assert rel_l2(to_grid(out, perm), ref) <= TOL[torch.float32], op
