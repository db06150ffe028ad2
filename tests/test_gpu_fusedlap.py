"""Single-pass Laplacian (NB_LAP_FUSED): each tile stages f on its nodes and
two rings of neighbours and computes the gradient on its nodes and the first
ring in shared memory, then the divergence of it.  Every output has the
arithmetic of the two-pass route, so the fused results equal the two-pass
ones bit for bit, and meet the oracle gates."""
import numpy as np
import pytest
import torch

import oracle
from paper_1908_06091_b300 import nabla
from gpu_helpers import (error_stats, inputs, oracle_mesh, oracle_op, pole_mask, product, rel_l2, to_device,
                         to_grid)

pytestmark = pytest.mark.gpu


def _lap(meth, fs, fd, route, grad_too):
    meth.set_laplacian_route(route)
    try:
        lap = fs.create_field(fill=float("nan"))
        if grad_too:
            g = fs.create_field(nvar=2, fill=float("nan"))
            nabla.gradlap(meth, fd, g, lap)
        else:
            g = None
            nabla.laplacian(meth, fd, lap)
        torch.cuda.synchronize()
        assert nabla.device_status() == 0
    finally:
        meth.set_laplacian_route(nabla.LAP_TWO_PASS)
    return g, lap


@pytest.mark.parametrize("N,nlev", [(16, 16), (32, 37), (32, 137), (48, 91), (24, 20)])
@pytest.mark.parametrize("grad_too", [False, True], ids=["lap", "gradlap"])
def test_fused_route_equals_two_pass_bitwise(N, nlev, grad_too):
    g_, m, meth = product(N)
    om = oracle_mesh(N)
    f, _ = inputs(om, nlev, 10, torch.float32)
    fs = nabla.NodeColumns(meth, nlev, torch.float32)
    fd = to_device(fs, f, m.permutation(), 1)
    before = nabla.launch_count()
    g1, l1 = _lap(meth, fs, fd, nabla.LAP_FUSED, grad_too)
    fused_launches = nabla.launch_count() - before
    g2, l2 = _lap(meth, fs, fd, nabla.LAP_TWO_PASS, grad_too)
    lv = slice(0, nlev)
    assert torch.equal(l1[:, lv], l2[:, lv])
    if grad_too:
        assert torch.equal(g1[:, lv], g2[:, lv])
    assert fused_launches <= 2  # one fused launch (plus the plan's record fill on first use)
    ref = oracle_op(om, "lap", f.astype(np.float64))
    assert rel_l2(to_grid(l1, m.permutation()), ref) <= 1e-5


def test_fused_route_o320_137_levels_against_the_oracle():
    """O320 x 137 (several hundred tiles, pole tiles, ragged last level
    unit): relative-L2, per-node maximum and pole-row gates."""
    N, nlev = 320, 137
    g_, m, meth = product(N)
    om = oracle_mesh(N)
    f, _ = inputs(om, nlev, 40, torch.float32)
    fs = nabla.NodeColumns(meth, nlev, torch.float32)
    perm = m.permutation()
    fd = to_device(fs, f, perm, 1)
    g, lap = _lap(meth, fs, fd, nabla.LAP_FUSED, True)
    pole = pole_mask(om)
    for out, op in ((lap, "lap"), (g, "grad")):
        s = error_stats(to_grid(out, perm), oracle_op(om, op, f.astype(np.float64)), pole)
        print(op, s)
        assert s["rel_l2"] <= 1e-5 and s["max_rel"] <= 1e-5 and s["pole_rel_l2"] <= 1e-5, (op, s)
    g2, l2 = _lap(meth, fs, fd, nabla.LAP_TWO_PASS, True)
    assert torch.equal(lap, l2) and torch.equal(g, g2)


@pytest.mark.parametrize("grid", ["F24", "PL"])
def test_fused_route_on_other_reduced_gaussian_grids(grid):
    pl = [20, 27, 33, 40, 44, 47, 47, 44, 40, 33, 27, 20] if grid == "PL" else None
    g = nabla.Grid.regular(24) if grid == "F24" else nabla.Grid.reduced(pl)
    m = nabla.Mesh(g, 1)
    meth = nabla.Method(m)
    nlev = 37
    fs = nabla.NodeColumns(meth, nlev, torch.float32)
    f = fs.create_field()
    f.copy_(torch.randn(f.shape, device="cuda", generator=torch.Generator(device="cuda").manual_seed(5)))
    g1, l1 = _lap(meth, fs, f, nabla.LAP_FUSED, True)
    g2, l2 = _lap(meth, fs, f, nabla.LAP_TWO_PASS, True)
    assert torch.equal(l1[:, :nlev], l2[:, :nlev]) and torch.equal(g1[:, :nlev], g2[:, :nlev])


def test_fused_route_leaves_fp64_and_short_columns_to_two_passes():
    g_, m, meth = product(16)
    for dtype, nlev in ((torch.float64, 37), (torch.float32, 7)):
        fs = nabla.NodeColumns(meth, nlev, dtype)
        f = fs.create_field()
        f.copy_(torch.randn(f.shape, dtype=dtype, device="cuda"))
        _, l1 = _lap(meth, fs, f, nabla.LAP_FUSED, False)
        _, l2 = _lap(meth, fs, f, nabla.LAP_TWO_PASS, False)
        assert torch.equal(l1, l2)
    with pytest.raises(nabla.NablaError):
        meth.set_laplacian_route(7)


def test_fused_route_wait_that_runs_out_reports_timeout():
    g_, m, meth = product(320)
    nlev = 137
    fs = nabla.NodeColumns(meth, nlev, torch.float32)
    f = fs.create_field()
    f.copy_(torch.randn(f.shape, device="cuda", generator=torch.Generator(device="cuda").manual_seed(9)))
    _lap(meth, fs, f, nabla.LAP_FUSED, False)  # plan built
    assert nabla.device_status(clear=True) == 0
    meth.set_wait_limit(0)
    meth.set_laplacian_route(nabla.LAP_FUSED)
    try:
        lap = fs.create_field(fill=float("nan"))
        nabla.laplacian(meth, f, lap)
        torch.cuda.synchronize()
        assert nabla.device_status(clear=True) == nabla.NB_ETIMEOUT
    finally:
        meth.set_wait_limit(-1)
        meth.set_laplacian_route(nabla.LAP_TWO_PASS)
    _, l1 = _lap(meth, fs, f, nabla.LAP_FUSED, False)
    _, l2 = _lap(meth, fs, f, nabla.LAP_TWO_PASS, False)
    assert torch.equal(l1, l2)
