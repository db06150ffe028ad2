"""The bounds-checked build (-DNB_BOUNDS_CHECK, loaded with NB_LIBRARY=debug):
its kernels check every gathered index (CSR neighbours, halo nodes, staged
column offsets, tile geometry) and record NB_EINVAL in the device status
word instead of reading outside a buffer.  On valid inputs it must give
oracle-correct results with the status word at 0.  The failure branch is
exercised on the host only (corrupted plans refused before upload,
tests/test_capi_host.py); no corrupted index is run on the GPU."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def test_bounds_checked_build_gives_oracle_results_and_a_clean_status():
    from paper_1908_06091_b300 import build
    lib = build.build(variant="debug")
    assert os.path.exists(lib)
    env = dict(os.environ, NB_LIBRARY="debug")
    r = subprocess.run([sys.executable, os.path.join(HERE, "_debug_build_cases.py")], env=env, cwd=ROOT,
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    res = json.loads(r.stdout.strip().splitlines()[-1])
    assert "bounds-checked" in res["version"]
    assert res["status"] == 0
    assert res["worst"]["f32"] <= 1e-5 and res["worst"]["f64"] <= 1e-12, res
