"""The odd-shape parity suites under the bounds-checked build.

The library compiled with SFSEG_DEBUG (libsfseg_debug.so) checks every work
item's range, the TMA box coordinates, the plan slots and the store offsets
inside the kernels, recording a violation instead of making the access.  This
test reruns the odd-shape, batched, fused and split-video parity tests in a
fresh process on that build (SFSEG_LIBRARY=debug); the conftest fixture there
asserts that each test left no violation, and the tests themselves still
compare with the oracle."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SUITES = ["tests/test_gpu_parity.py", "tests/test_gpu_fused.py", "tests/test_gpu_slab.py",
          "tests/test_gpu_multichannel.py", "tests/test_gpu_cluster.py"]


def test_parity_suites_under_the_bounds_checked_build(cuda_device):
    env = dict(os.environ, SFSEG_LIBRARY="debug")
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-m", "gpu", "-p", "no:cacheprovider",
                        *SUITES], cwd=ROOT, env=env, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-4000:] + r.stderr[-2000:]
    assert " passed" in r.stdout
