import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: takes more than a few seconds")


GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


@pytest.fixture
def golden_dir():
    return GOLDEN


def _ensure_library():
    """Build libqtc.so in-tree if it is missing (nvcc cross-compiles on CPU)."""
    lib = os.path.join(ROOT, "paper_1709_03636_gb300", "libqtc.so")
    if not os.path.exists(lib):
        import importlib.util
        path = os.path.join(ROOT, "paper_1709_03636_gb300", "build.py")
        spec = importlib.util.spec_from_file_location("_qtc_build", path)
        mod = importlib.util.module_from_spec(spec)
        spec.loader.exec_module(mod)
        mod.build()


_ensure_library()
