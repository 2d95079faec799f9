import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    # the batch autotuner's persistent cache: tests keep theirs apart from a
    # user's (and from a benchmark run after them)
    import tempfile
    os.environ.setdefault("AP_TUNE_CACHE", os.path.join(tempfile.mkdtemp(prefix="alnplot-tests-"), "tune.txt"))
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (runs the CUDA path)")
    config.addinivalue_line("markers", "slow: long-running CPU test")


def gpu_available() -> bool:
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:  # pragma: no cover
        return False


@pytest.fixture(scope="session")
def cuda_lib():
    """The built CUDA library binding; fails loudly if it cannot load."""
    if not gpu_available():
        pytest.fail("GPU test selected but no CUDA device is visible")
    import paper_0909_2000_gb300 as ap
    ap.load()
    return ap
