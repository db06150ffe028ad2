"""Host checks of bench.py's roofline arithmetic (no GPU).

The algorithmic bytes of a launch follow from what it must move: every
input value read once, every output value written once, and the CSR and
FP32 weights read once per node.  These tests restate that count from the
mesh sizes (V = 4N^2 + 36N nodes of O<N>, E = 3V - 6 edges) and check the
bench's figures and the DRAM-traffic record against it.
"""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def sizes(N):
    V = 4 * N * N + 36 * N
    return V, 3 * V - 6


def test_benchmark_mesh_sizes():
    V, E = sizes(1280)
    assert (V, E) == (6_599_680, 19_799_034)


@pytest.mark.parametrize("N,L", [(1280, 137), (320, 137), (32, 1)])
def test_algorithmic_bytes_per_launch(N, L):
    V, E = sizes(N)
    P = 2 * E  # CSR entries
    # grad: a scalar in (4 B), two components out (8 B); per CSR entry an
    # index (4 B) and the (gx, gy) weight pair (8 B); V + 1 row pointers
    assert bench.algorithmic_bytes("grad", V, E, L, 4) == 12 * V * L + 4 * (V + 1) + 12 * P
    # div or curl: a wind in (8 B), one scalar out (4 B), plus 8 B of self
    # weights per node
    assert bench.algorithmic_bytes("div", V, E, L, 4) == 12 * V * L + 4 * (V + 1) + 12 * P + 8 * V
    # fused div + curl: the wind read once, two scalars out, both weight pairs
    # (16 B per entry) and both self-weight pairs (16 B per node)
    assert bench.algorithmic_bytes("divcurl", V, E, L, 4) == 16 * V * L + 4 * (V + 1) + 20 * P + 16 * V
    # FP64 doubles every field and weight byte, not the CSR
    assert bench.algorithmic_bytes("grad", V, E, L, 8) == 24 * V * L + 4 * (V + 1) + 20 * P


def test_benchmark_figures():
    """The O1280 x 137 FP32 figures quoted with the measurements."""
    V, E = sizes(1280)
    gb = {op: bench.algorithmic_bytes(op, V, E, 137, 4) / 1e9 for op in ("grad", "div", "divcurl")}
    assert round(gb["grad"], 2) == 11.35
    assert round(gb["div"], 2) == 11.40
    assert round(gb["divcurl"], 2) == 15.39


def test_dram_traffic_record_is_near_the_algorithmic_bytes():
    """The ncu record, when it matches the kernel source, lies within a few
    per cent of the algorithmic bytes at the benchmark size: halo columns
    are re-read from L2, not from DRAM."""
    V, E = sizes(1280)
    L = 137
    for op in ("grad", "div", "divcurl"):
        t = bench.measured_traffic(op, V, L)
        if t is None:
            pytest.skip("the staged kernel changed since the DRAM record was taken")
        a = bench.algorithmic_bytes(op, V, E, L, 4)
        assert 0.9 * a < t < 1.1 * a, op


def test_defaults_keep_the_timing_rules(monkeypatch):
    monkeypatch.setattr(sys, "argv", ["bench.py"])
    a = bench.parse()
    assert a.warmup >= 3 and a.steps >= 1
    assert a.grid == 1280 and a.nlev == 137 and a.gpus == 1
    assert bench.FP64_PEAK_TFLOPS == 1.25


def test_cpu_baseline_reports_errors_against_the_oracle():
    """The CPU-baseline leg times the oracle on the run's own sampled inputs
    and reports the GPU outputs' error figures against it.  Here the 'GPU'
    outputs are the oracle's own (rounded to FP32) and a copy with one
    planted error, so the figures are known."""
    import types

    import numpy as np

    import oracle
    N, L = 16, 3
    m = oracle.build_mesh(N)
    rng = np.random.default_rng(0)
    f = rng.standard_normal((m.V, L))
    uv = rng.standard_normal((m.V, L, 2))
    exact = {"grad": oracle.grad(m, f), "div": oracle.div(m, uv), "curl": oracle.curl(m, uv),
             "lap": oracle.lap(m, f)}
    planted = dict(exact)
    planted["div"] = exact["div"].copy()
    planted["div"][0, 1] += 1.0  # a pole-row node (the first grid row)
    sample = {"levels": [0, 1, 2], "f": f, "uv": uv,
              "out32": {k: v.astype(np.float32) for k, v in exact.items()}, "out64": planted}
    cb, err = bench.cpu_baseline(types.SimpleNamespace(grid=N, nlev=L), sample)
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] > 0
    assert cb["single_core"]["value"] > 0
    for op in ("grad", "div", "curl", "lap"):
        assert err["f32"][op]["rel_l2"] < 1e-6 and err["f32"][op]["max_rel"] < 1e-6
        assert err["f64"][op]["max_abs"] == (1.0 if op == "div" else 0.0)
    assert err["f64"]["div"]["pole_rel_l2"] > 0
    assert err["f64"]["div"]["max_rel"] == pytest.approx(1.0 / np.abs(exact["div"]).max(), rel=1e-3)
