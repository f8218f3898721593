import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built libset.so")
    config.addinivalue_line("markers", "slow: long-running CPU test")
    # incremental in-tree build of libset.so (seconds when up to date) before any test imports it
    import importlib.util
    spec = importlib.util.spec_from_file_location("set_build", os.path.join(ROOT, "paper_2606_05495_gb300", "build.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    mod.build()


@pytest.fixture(scope="session")
def golden_dir():
    return os.path.join(ROOT, "tests", "golden")
