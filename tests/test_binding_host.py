"""Host-side checks of the Python binding (no GPU): every entry point that takes matrices
rejects anything but a 2-D float64 CUDA tensor before it reaches the library, so no CPU
path exists behind the binding."""
import numpy as np
import pytest
import torch

import paper_0912_2572_gb300 as ts
from paper_0912_2572_gb300 import build


@pytest.fixture(scope="module", autouse=True)
def built():
    build.build()


def host_matrices():
    a = torch.zeros((64, 4), dtype=torch.float64)
    return [a, a.float(), a.numpy(), np.zeros((64, 4)), a[:, 0]]


@pytest.mark.parametrize("bad", host_matrices(), ids=["cpu_f64", "cpu_f32", "numpy_view", "numpy", "1d"])
def test_entry_points_reject_host_matrices(bad):
    with pytest.raises(TypeError):
        ts.factor(bad)
    with pytest.raises(TypeError):
        ts.factor(bad, qt=bad)
    with pytest.raises(TypeError):
        ts.orthonormalize(bad)
    with pytest.raises(TypeError):
        ts.orthonormalize(bad, Q=bad)
    with pytest.raises(TypeError):
        ts.lstsq(bad, bad)
    with pytest.raises(TypeError):
        ts.factor_autotune(bad)
