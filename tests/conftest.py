import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built libtsqr.so")
    config.addinivalue_line("markers", "slow: long-running case")


def _has_gpu():
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


def pytest_collection_modifyitems(config, items):
    if _has_gpu():
        return
    skip = pytest.mark.skip(reason="no CUDA GPU in this environment")
    for item in items:
        if "gpu" in item.keywords:
            item.add_marker(skip)


@pytest.fixture(scope="session")
def cuda_lib():
    """The built CUDA library (built on first use if missing) on cuda:0."""
    import torch
    from paper_0912_2572_gb300 import build, _lib
    build.build()
    torch.cuda.set_device(0)
    return _lib.load()


def to_dev(a):
    """NumPy column-major float64 -> column-major CUDA tensor (same bytes)."""
    import torch
    a = np.asarray(a, dtype=np.float64)
    if a.ndim == 1:
        a = a.reshape(-1, 1)
    return torch.from_numpy(np.ascontiguousarray(a.T)).cuda().t()


def to_host(t):
    return t.cpu().numpy()
