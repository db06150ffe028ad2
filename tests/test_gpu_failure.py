"""Failure detection on the GPU without a fault.

The staged kernels bound every wait of their copy pipeline.  A wait limit of
zero (nb_method_set_wait_limit) makes each wait test its barrier once: a
consumer warp that finds its CTA's first tile not yet copied gives up, the
kernel records NB_ETIMEOUT in the device status word, every CTA waits for
the copies it has issued, and the kernel returns.  No wait is left
unbounded, nothing faults, and the context stays usable: the next call with
the default limit is correct against the oracle."""
import numpy as np
import pytest
import torch

from paper_1908_06091_b300 import nabla
from gpu_helpers import inputs, oracle_mesh, oracle_op, product, rel_l2, run_op, to_device, to_grid

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("op", ["grad", "divcurl"])
def test_wait_that_runs_out_reports_timeout_and_the_next_call_is_correct(op):
    N, nlev = 320, 137  # FP32, >= 16 levels, aligned: the staged kernels
    g, m, meth = product(N)
    om = oracle_mesh(N)
    f, uv = inputs(om, nlev, 10, torch.float32)
    perm = m.permutation()
    fs = nabla.NodeColumns(meth, nlev, torch.float32)
    x = to_device(fs, f if op == "grad" else uv, perm, 1 if op == "grad" else 2)
    assert nabla.device_status(clear=True) == 0

    def call():
        outs = ([fs.create_field(nvar=2, fill=float("nan"))] if op == "grad"
                else [fs.create_field(fill=float("nan")), fs.create_field(fill=float("nan"))])
        before = nabla.launch_count()
        if op == "grad":
            nabla.apply(meth, "grad", x, outs[0])
        else:
            nabla.divcurl(meth, x, outs[0], outs[1])
        assert nabla.launch_count() == before + 1  # one staged launch
        torch.cuda.synchronize()
        return outs

    meth.set_wait_limit(0)
    try:
        call()
        assert nabla.device_status(clear=True) == nabla.NB_ETIMEOUT
    finally:
        meth.set_wait_limit(-1)
    outs = call()
    assert nabla.device_status() == 0
    if op == "grad":
        assert rel_l2(to_grid(outs[0], perm), oracle_op(om, "grad", f.astype(np.float64))) <= 1e-5
    else:
        for t, o in zip(outs, ("div", "curl")):
            assert rel_l2(to_grid(t, perm), oracle_op(om, o, uv.astype(np.float64))) <= 1e-5


def test_wait_limit_argument_is_checked():
    g, m, meth = product(16)
    for bad in (-2, 60_000_000_001):
        with pytest.raises(nabla.NablaError):
            meth.set_wait_limit(bad)
    meth.set_wait_limit(5_000_000)
    meth.set_wait_limit(-1)
