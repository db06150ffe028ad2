"""The C ABI from plain C: compile tests/c/capi_host_client.c with gcc
(-std=c99 -pedantic) against include/nabla_b300.h, link the library, and run
its host-side checks (grid, mesh, CSR, permutation, EqualRegions partition
and one-ring halos).  No GPU is needed."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
LIBDIR = os.path.join(ROOT, "paper_1908_06091_b300", "_lib")
SRC = os.path.join(ROOT, "tests", "c", "capi_host_client.c")


@pytest.fixture(scope="module")
def client(tmp_path_factory):
    if not os.path.exists(os.path.join(LIBDIR, "libnabla_b300.so")):
        pytest.fail("libnabla_b300.so is not built (run __graft_entry__.build())")
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    exe = str(tmp_path_factory.mktemp("capi") / "capi_host_client")
    subprocess.run(["gcc", "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", "-O2",
                    "-I" + os.path.join(ROOT, "include"), SRC, "-L" + LIBDIR, "-lnabla_b300",
                    "-Wl,-rpath," + LIBDIR, "-o", exe], check=True)
    return exe


@pytest.mark.parametrize("N,nparts", [(16, 2), (32, 4), (32, 7)])
def test_c_client_host_calls(client, N, nparts):
    r = subprocess.run([client, str(N), str(nparts)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "failures 0" in r.stdout
