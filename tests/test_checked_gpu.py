"""The checked build (libgsr_checked.so: GSR_CHECKED device-side index checks
that record GSR_EINTERNAL instead of trapping -- the stand-in for a memory
sanitizer): a subset of the parity suite runs against it in a child process
and must pass with every status word clean."""
import os
import subprocess
import sys

import pytest
import torch

from paper_2411_17660_b300 import build

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def test_parity_subset_on_the_checked_build():
    lib = build.build(checked=True)
    env = dict(os.environ, GSR_LIBRARY=lib)
    which = subprocess.run([sys.executable, "-c", "from paper_2411_17660_b300 import binding as B; B.load(); "
                            "print(B.LIB_PATH)"], env=env, cwd=ROOT, capture_output=True, text=True, timeout=300)
    assert which.returncode == 0 and which.stdout.strip() == lib, which.stderr[-2000:]
    r = subprocess.run([sys.executable, "-m", "pytest", "tests/test_parity_gpu.py", "tests/test_binning_gpu.py",
                        "tests/test_surfel_gpu.py", "-q", "-x", "-p", "no:cacheprovider", "-m", "gpu", "-k",
                        "reduced or strategies or capacity or surfel or tiny or decisions"],
                       env=env, cwd=ROOT, capture_output=True, text=True, timeout=1500)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-2000:]
