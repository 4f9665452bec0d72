import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the compiled library")
    config.addinivalue_line("markers", "slow: full-size case (minutes)")


@pytest.fixture(scope="session")
def tiny_workload():
    from paper_2605_20565_gb300 import synth
    return synth.tiny()


@pytest.fixture(scope="session")
def tiny_tree(tiny_workload):
    import oracle
    w = tiny_workload
    return oracle.octree_build(w.spheres, w.lmin, w.lmax)
