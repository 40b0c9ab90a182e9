"""The allocation-free least-squares entry point, tsqr_lstsq_static.

It exists for callers that cannot allocate device memory when they need a solve: code
running in host callbacks, plugins whose framework owns every allocation, or programs
that reserve the whole GPU at start-up and forbid later cudaMalloc calls. Instead of
allocating, it keeps its scratch in a fixed 64 MiB device array inside the library.

These tests call it through the C ABI with caller-owned buffers and check, on two calls
in a row with different problems (so stale contents of the shared array would show),
that its solution matches tsqr_lstsq's within the least-squares tolerance of the other
GPU tests, that a repeat call does not change the device's free memory, and that a
problem too large for the array is refused before any work is enqueued.
"""
import ctypes

import numpy as np
import pytest

import oracle
from paper_0912_2572_gb300 import inputs
from conftest import to_dev, to_host

pytestmark = pytest.mark.gpu

TOL = 1e-12  # the least-squares tolerance of the well-conditioned GPU parity tests


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def _static(lib, Ad, Bd, Xd, stream):
    m, n = Ad.shape
    k = Bd.shape[1]
    return lib.tsqr_lstsq_static(Ad.data_ptr(), m, n, Ad.stride(1), Bd.data_ptr(), m, k, Xd.data_ptr(),
                                 Xd.stride(1), stream)


def _reference(lib, Ad, Bd, stream):
    import torch
    import paper_0912_2572_gb300 as ts
    m, n = Ad.shape
    k = Bd.shape[1]
    leaf_h = ts.plan_describe(m, n, 4096, 2, True, nc=n + k)["tile_rows"]
    X = torch.empty((k, n), dtype=torch.float64, device="cuda").t()
    st = lib.tsqr_lstsq(Ad.data_ptr(), m, n, Ad.stride(1), Bd.data_ptr(), m, k, X.data_ptr(), n, leaf_h, 2, 0,
                        2, 0, stream, None)
    assert st == 0
    return X


def test_static_matches_lstsq_on_two_calls(cuda_lib):
    import torch
    lib = cuda_lib
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    cases = [(100_000, 32, 3, 21), (50_000, 64, 1, 22)]
    prepared = []
    for m, n, k, seed in cases:
        A = inputs.gaussian(m, n, seed)
        B, _ = inputs.lstsq_rhs(A, k, 1e-3, seed + 100)
        Ad, Bd = to_dev(A), to_dev(B)
        Xd = torch.full((k, n), float("nan"), dtype=torch.float64, device="cuda").t()
        Xref = _reference(lib, Ad, Bd, stream)
        prepared.append((A, B, Ad, Bd, Xd, Xref))
    torch.cuda.synchronize()
    for i, (A, B, Ad, Bd, Xd, Xref) in enumerate(prepared):
        free_before = torch.cuda.mem_get_info()[0]
        assert _static(lib, Ad, Bd, Xd, stream) == 0
        torch.cuda.synchronize()
        free_after = torch.cuda.mem_get_info()[0]
        if i > 0:  # the first call may load the module that holds the static array
            assert free_after == free_before
        X = to_host(Xd)
        assert np.all(np.isfinite(X))
        assert rel(X, to_host(Xref)) <= TOL
        assert rel(X, oracle.lstsq(A, B)) <= TOL
        assert np.array_equal(to_host(Bd), B)  # the caller's B is untouched


def test_static_single_tile_and_singular(cuda_lib):
    """A problem shorter than one on-chip tile (a one-job plan with no tree) against the
    oracle, a square problem, then an A with a zero column: R then has an exactly zero
    diagonal entry and the call reports TSQR_ERR_SINGULAR with a message."""
    import torch
    lib = cuda_lib
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for m, n, k, seed in ((100, 8, 2, 31), (24, 24, 1, 32)):
        A = inputs.gaussian(m, n, seed)
        B = inputs.gaussian(m, k, seed + 1)
        Ad, Bd = to_dev(A), to_dev(B)
        Xd = torch.full((k, n), float("nan"), dtype=torch.float64, device="cuda").t()
        assert _static(lib, Ad, Bd, Xd, stream) == 0
        torch.cuda.synchronize()
        assert lib.tsqr_last_error() == b""
        assert rel(to_host(Xd), oracle.lstsq(A, B)) <= (1e-10 if m == n else TOL)
    A = inputs.gaussian(3000, 6, 33)
    A[:, 2] = 0.0
    B = inputs.gaussian(3000, 1, 34)
    Xd = torch.zeros((1, 6), dtype=torch.float64, device="cuda").t()
    assert _static(lib, to_dev(A), to_dev(B), Xd, stream) == 4
    assert b"zero diagonal" in lib.tsqr_last_error()


def test_static_refuses_oversized_problem(cuda_lib):
    import torch
    lib = cuda_lib
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    # 2,000,000 x 64 needs about 1 GB of scratch: refused, nothing enqueued
    st = lib.tsqr_lstsq_static(4096, 2_000_000, 64, 2_000_000, 4096, 2_000_000, 1, 4096, 64, stream)
    assert st == 6
    assert b"exceeds" in lib.tsqr_last_error()
    assert lib.tsqr_lstsq_static(None, 10, 2, 10, 4096, 10, 1, 4096, 2, stream) == 1
    assert lib.tsqr_last_error() != b""
    assert lib.tsqr_lstsq_static(4096, 10, 100, 10, 4096, 10, 40, 4096, 100, stream) == 1
