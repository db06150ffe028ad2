"""Parity cases run with the bounds-checked build (NB_LIBRARY=debug), in a
process of their own: every operator on the direct and the staged kernels,
the fused calls, the single-pass Laplacian and a batch, on O32 and O48.
Prints one JSON line: the library version, the device status word after all
cases, and the worst relative L2 error against the oracle per dtype."""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))
sys.path.insert(0, HERE)

import numpy as np  # noqa: E402
import torch  # noqa: E402

from paper_1908_06091_b300 import nabla  # noqa: E402
from gpu_helpers import inputs, oracle_mesh, oracle_op, product, rel_l2, to_device, to_grid  # noqa: E402

assert os.environ.get("NB_LIBRARY") == "debug"
worst = {"f32": 0.0, "f64": 0.0}
for N, nlev in ((32, 37), (48, 20), (32, 137)):
    g, m, meth = product(N)
    om = oracle_mesh(N)
    perm = m.permutation()
    for dtype, key in ((torch.float32, "f32"), (torch.float64, "f64")):
        f, uv = inputs(om, nlev, 10, dtype)
        fs = nabla.NodeColumns(meth, nlev, dtype)
        fd, uvd = to_device(fs, f, perm, 1), to_device(fs, uv, perm, 2)
        refs = {op: oracle_op(om, op, (f if op in ("grad", "lap") else uv).astype(np.float64))
                for op in ("grad", "div", "curl", "lap")}
        for variant in (nabla.KERNEL_DIRECT, nabla.KERNEL_AUTO):
            meth.set_kernel(variant)
            for op in ("grad", "div", "curl", "lap"):
                out = fs.create_field(nvar=2 if op == "grad" else 1, fill=float("nan"))
                nabla.apply(meth, op, fd if op in ("grad", "lap") else uvd, out)
                torch.cuda.synchronize()
                worst[key] = max(worst[key], rel_l2(to_grid(out, perm), refs[op]))
        meth.set_kernel(nabla.KERNEL_AUTO)
        d, z = fs.create_field(), fs.create_field()
        nabla.divcurl(meth, uvd, d, z)
        for route in (nabla.LAP_TWO_PASS, nabla.LAP_FUSED):
            meth.set_laplacian_route(route)
            gg, ll = fs.create_field(nvar=2), fs.create_field()
            nabla.gradlap(meth, fd, gg, ll)
            torch.cuda.synchronize()
            worst[key] = max(worst[key], rel_l2(to_grid(ll, perm), refs["lap"]),
                             rel_l2(to_grid(gg, perm), refs["grad"]))
        meth.set_laplacian_route(nabla.LAP_TWO_PASS)
        torch.cuda.synchronize()
        worst[key] = max(worst[key], rel_l2(to_grid(d, perm), refs["div"]), rel_l2(to_grid(z, perm), refs["curl"]))
        # a batch of the four operators (persistent and staged routes)
        items = []
        for op in ("grad", "div", "curl", "lap"):
            items.append((op, meth, fd if op in ("grad", "lap") else uvd,
                          fs.create_field(nvar=2 if op == "grad" else 1, fill=float("nan"))))
        b = nabla.Batch(items)
        b.run()
        torch.cuda.synchronize()
        for op, _, _, out in items:
            worst[key] = max(worst[key], rel_l2(to_grid(out, perm), refs[op]))
print(json.dumps({"version": nabla.version(), "status": nabla.device_status(), "worst": worst}))
