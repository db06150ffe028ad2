"""GPU parity on the other grid families: the regular F<N> grid (Sec.
4.2.3.6) and a PL-array grid with odd pole rings (Sec. 4.2.3.7), all four
operators and the fused div+curl against the FP64 oracle."""
import functools

import numpy as np
import pytest
import torch

import oracle
from paper_1908_06091_b300 import nabla
from gpu_helpers import R, inputs, oracle_op, rel_l2, run_op, to_device, to_grid

pytestmark = pytest.mark.gpu

TOL = {torch.float64: 1e-12, torch.float32: 1e-5}


def _pl(kind, N):
    if kind == "F":
        return oracle.regular_nx(N)
    o = oracle.row_nx(N)
    pl = (np.round(o * 1.1 / 5) * 5 + (np.arange(2 * N) % 3 == 0)).astype(np.int32)
    pl[N:] = pl[:N][::-1]
    return pl


@functools.lru_cache(maxsize=4)
def _both(kind, N):
    pl = _pl(kind, N)
    g = nabla.Grid.regular(N) if kind == "F" else nabla.Grid.reduced(pl)
    m = nabla.Mesh(g, 1)
    return g, m, nabla.Method(m, R), oracle.build_mesh(N, R, pl=pl)


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64], ids=["f32", "f64"])
@pytest.mark.parametrize("kind,N,nlev", [("F", 32, 1), ("F", 32, 137), ("P", 32, 37), ("P", 64, 137)])
def test_all_operators_meet_the_gate(kind, N, nlev, dtype):
    g, m, meth, om = _both(kind, N)
    f, uv = inputs(om, nlev, 10, dtype)
    perm = m.permutation()
    fs = nabla.NodeColumns(meth, nlev, dtype)
    fd, uvd = to_device(fs, f, perm, 1), to_device(fs, uv, perm, 2)
    for op in ("grad", "div", "curl", "lap"):
        x, xh = (fd, f) if op in ("grad", "lap") else (uvd, uv)
        got = to_grid(run_op(meth, fs, op, x), perm)
        err = rel_l2(got, oracle_op(om, op, xh.astype(np.float64)))
        assert err <= TOL[dtype], (kind, N, nlev, op, err)
    d, z = fs.create_field(fill=float("nan")), fs.create_field(fill=float("nan"))
    nabla.divcurl(meth, uvd, d, z)
    torch.cuda.synchronize()
    lv = slice(0, nlev)  # padding levels hold NaN on both sides
    assert torch.equal(d[:, lv], run_op(meth, fs, "div", uvd)[:, lv])
    assert torch.equal(z[:, lv], run_op(meth, fs, "curl", uvd)[:, lv])
    assert nabla.device_status() == 0
