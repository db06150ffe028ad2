import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_sessionstart(session):
    """Build the CUDA library and the oracle in-tree if they are missing or stale."""
    from paper_1908_06091_b300 import build as lib_build
    import oracle
    lib_build.build()
    oracle.build()


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (B300) and the built CUDA library")
    config.addinivalue_line("markers", "slow: larger CPU cases")


_MESHES = {}


def oracle_mesh(N):
    """Session cache of oracle meshes (built with no planted mistake)."""
    import oracle
    if N not in _MESHES:
        assert oracle.lib().or_get_mutation() == 0
        _MESHES[N] = oracle.build_mesh(N)
    return _MESHES[N]


@pytest.fixture(scope="session")
def mesh_factory():
    return oracle_mesh

TESTS = os.path.dirname(os.path.abspath(__file__))
if TESTS not in sys.path:
    sys.path.insert(0, TESTS)
