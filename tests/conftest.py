import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU; calls the CUDA path through the C-ABI")
    config.addinivalue_line("markers", "slow: long-running CPU test")


@pytest.fixture(scope="session")
def cuda_device():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


@pytest.fixture(autouse=True)
def _debug_build_clean(request):
    """Under the bounds-checked build (SFSEG_LIBRARY=debug) every GPU test must
    leave no recorded violation (item ranges, TMA coordinates, workspace
    offsets)."""
    yield
    if os.environ.get("SFSEG_LIBRARY") != "debug" or request.node.get_closest_marker("gpu") is None:
        return
    import paper_1907_02731_gb300 as sf
    assert sf.load_library().sfseg_debug_build() == 1
    n, code, vals = sf.sfseg_debug_status()
    assert n == 0, f"debug build: {n} bounds violations, first code {code} values {vals}"
