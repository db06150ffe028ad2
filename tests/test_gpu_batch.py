"""Batched launch (CUDA graph) against single-op runs.

An item on the persistent-kernel route must equal the same operation run
alone on the direct kernels bit for bit (same per-point arithmetic); an item
on the staged route (levels-per-block 0) must equal the operation run alone
with the default kernel choice.  This holds before and after autotuning, and
FP32 results also meet the oracle gate."""
import os

import numpy as np
import pytest
import torch

from paper_1908_06091_b300 import nabla
from gpu_helpers import inputs, oracle_mesh, oracle_op, product, rel_l2, to_device, to_grid

pytestmark = pytest.mark.gpu


def _mixed_items(seed=3):
    rng = np.random.default_rng(seed)
    items, meta = [], []
    for N in (16, 24, 32):
        g, m, meth = product(N)
        om = oracle_mesh(N)
        perm = m.permutation()
        for nlev in (1, 5, 37):
            for dtype in (torch.float32, torch.float64):
                f, uv = inputs(om, nlev, 10, dtype, seed=int(rng.integers(1 << 30)))
                fs = nabla.NodeColumns(meth, nlev, dtype)
                for op in ("grad", "div", "curl", "lap"):
                    x = to_device(fs, f if op in ("grad", "lap") else uv, perm, 1 if op in ("grad", "lap") else 2)
                    out = fs.create_field(nvar=2 if op == "grad" else 1, fill=float("nan"))
                    items.append((op, meth, x, out))
                    meta.append((N, nlev, dtype, op, fs, f if op in ("grad", "lap") else uv))
    return items, meta


def _single_direct(meth, fs, op, x, variant=nabla.KERNEL_DIRECT):
    meth.set_kernel(variant)
    out = fs.create_field(nvar=2 if op == "grad" else 1, fill=float("nan"))
    nabla.apply(meth, op, x, out)
    meth.set_kernel(nabla.KERNEL_AUTO)
    return out


def _single_for_route(meth, fs, op, x, lpb):
    return _single_direct(meth, fs, op, x, nabla.KERNEL_AUTO if lpb == 0 else nabla.KERNEL_DIRECT)


def test_batched_results_equal_single_ops_bitwise_and_meet_gate():
    items, meta = _mixed_items()
    b = nabla.Batch(items)
    b.run()
    torch.cuda.synchronize()
    assert nabla.device_status() == 0
    for (op, meth, x, out), (N, nlev, dtype, _, fs, xh) in zip(items, meta):
        ref = _single_direct(meth, fs, op, x)
        torch.cuda.synchronize()
        assert torch.equal(out, ref), (N, nlev, dtype, op)
    # spot-check the oracle gate on a few items
    for k in range(0, len(items), 7):
        (op, meth, x, out), (N, nlev, dtype, _, fs, xh) = items[k], meta[k]
        got = to_grid(out, product(N)[1].permutation())
        ref = oracle_op(oracle_mesh(N), op, xh.astype(np.float64))
        assert rel_l2(got, ref) <= (1e-5 if dtype == torch.float32 else 1e-12), (N, nlev, dtype, op)


def test_graph_replay_is_deterministic_and_tuning_keeps_results(tmp_path, monkeypatch):
    monkeypatch.setenv("NB_TUNE_CACHE", str(tmp_path / "tune.txt"))
    items, meta = _mixed_items(seed=5)
    b = nabla.Batch(items)
    b.run()
    torch.cuda.synchronize()
    first = [o.clone() for (_, _, _, o) in items]
    for _, _, _, o in items:
        o.fill_(float("nan"))
    b.run()
    torch.cuda.synchronize()
    assert all(torch.equal(a, o) for a, (_, _, _, o) in zip(first, items))
    before = b.info()
    b.tune()
    after = b.info()
    for _, _, _, o in items:
        o.fill_(float("nan"))
    b.run()
    torch.cuda.synchronize()
    for k, ((op, meth, x, o), m) in enumerate(zip(items, meta)):
        if after["levels_per_block"][k] == before["levels_per_block"][k] or \
                (after["levels_per_block"][k] > 0 and before["levels_per_block"][k] > 0):
            assert torch.equal(first[k], o), m[:4]  # same route: same bits
        ref = _single_for_route(meth, m[4], op, x, after["levels_per_block"][k])
        torch.cuda.synchronize()
        assert torch.equal(o, ref), m[:4]
    assert after["node_levels"] == before["node_levels"]
    assert set(after["nodes_per_warp"]) <= {0, 1, 2, 4, 8, 16, 32}
    assert set(after["levels_per_block"]) <= {0, 4, 8, 16, 32, 64}
    lines = (tmp_path / "tune.txt").read_text().strip().splitlines()
    assert len(lines) >= 1 and all(len(ln.split("|")) == 7 for ln in lines)


def test_batch_rejects_bad_items():
    g, m, meth = product(16)
    fs = nabla.NodeColumns(meth, 4, torch.float32)
    f = fs.create_field()
    with pytest.raises((nabla.NablaError, ValueError)):
        nabla.Batch([("grad", meth, f, fs.create_field())])  # grad output must be a vector
    g2, m2, meth2 = product(24)
    fs2 = nabla.NodeColumns(meth2, 4, torch.float32)
    with pytest.raises(nabla.NablaError):
        nabla.Batch([("grad", meth, fs2.create_field(), fs2.create_field(nvar=2))])


def test_large_items_take_the_staged_route_and_match_single_ops():
    """Items of a few million node-levels default to the staged kernels; a
    small item in the same batch stays on the persistent kernel."""
    items, meta = [], []
    for N, nlev, ops in ((96, 137, ("grad", "div", "curl", "lap")), (16, 5, ("lap",))):
        g, m, meth = product(N)
        om = oracle_mesh(N)
        f, uv = inputs(om, nlev, 10, torch.float32)
        fs = nabla.NodeColumns(meth, nlev, torch.float32)
        for op in ops:
            x = to_device(fs, f if op in ("grad", "lap") else uv, m.permutation(), 1 if op in ("grad", "lap") else 2)
            out = fs.create_field(nvar=2 if op == "grad" else 1, fill=float("nan"))
            items.append((op, meth, x, out))
            meta.append((N, nlev, op, fs))
    b = nabla.Batch(items)
    info = b.info()
    assert info["levels_per_block"][:4] == [0, 0, 0, 0] and info["levels_per_block"][4] > 0
    launches = nabla.launch_count()
    b.run()
    b.run()
    torch.cuda.synchronize()
    assert nabla.device_status() == 0
    assert nabla.launch_count() > launches
    # the captured graph: two persistent phases (the small Laplacian's
    # gradient and divergence), the staged launches (grad, div, curl and two
    # for the Laplacian), plus the counter reset and the fork / join
    g = b.info()
    assert g["graph_kernels"] == 2 + 3 + 2 and g["graph_nodes"] > g["graph_kernels"]
    for k, ((op, meth, x, out), (N, nlev, _, fs)) in enumerate(zip(items, meta)):
        ref = _single_for_route(meth, fs, op, x, info["levels_per_block"][k])
        torch.cuda.synchronize()
        assert torch.equal(out, ref), (N, nlev, op)
