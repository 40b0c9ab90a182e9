"""Mixed-precision least squares on the GPU: FP32 leaf factorizations, FP64 tree, FP64
refinement by corrected semi-normal equations (the paper has no mixed-precision
algorithm). The solution must match the FP64 oracle's to ||x - x_o|| / ||x_o|| <= 1e-10
for kappa(A) <= 1e4, with the corrections shrinking step by step."""
import numpy as np
import pytest

import oracle
from paper_0912_2572_gb300 import inputs
from conftest import to_dev, to_host

pytestmark = pytest.mark.gpu

TOL = 1e-10


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("m,n,k,dec,h,arity,two", [
    (4000, 16, 1, 4, 256, 2, True),
    (100_000, 32, 4, 4, 512, 2, True),
    (20_000, 64, 3, 3, 448, 4, False),
    (5000, 8, 10, 2, 128, 2, True),
    (3000, 100, 2, 4, 200, 2, True),
    (777, 5, 1, 4, 64, 0, False),
    (60_000, 128, 3, 4, 128, 2, True),
    (9000, 120, 9, 3, 256, 4, True),
])
def test_mixed_lstsq_matches_fp64_oracle(cuda_lib, m, n, k, dec, h, arity, two):
    import paper_0912_2572_gb300 as ts
    A = inputs.graded(m, n, dec)
    B, _ = inputs.lstsq_rhs(A, k, 1e-6, 5)
    X, hist = ts.lstsq(to_dev(A), to_dev(B), leaf_h=h, arity=arity, two_level=two, prec=ts.MIXED, max_refine=10,
                       info=True)
    X = to_host(X)
    Xo = oracle.lstsq(A, B)
    assert rel(X, Xo) <= TOL
    h = [v for v in hist if v > 0]
    assert len(h) >= 2 and h[0] == 1.0  # the first correction is the whole x
    assert all(b < a for a, b in zip(h[:-1], h[1:-1]))  # the last may sit at the rounding level
    # the stop: the predicted remaining correction (last x rho / (1 - rho), rho the largest
    # ratio of successive corrections) is below 1e-10, or the corrections stopped shrinking
    rho = max(b / a for a, b in zip(h[:-1], h[1:]))
    assert (rho < 0.5 and h[-1] * rho / (1 - rho) <= 1e-10) or (len(h) >= 3 and h[-1] > 0.5 * h[-2])


def test_mixed_needs_refinement_and_fp64_is_direct(cuda_lib):
    """With no correction step the FP32 factorization alone is far from FP64 accuracy at
    kappa = 1e4; the FP64 path is accurate without refinement."""
    import paper_0912_2572_gb300 as ts
    A = inputs.graded(50_000, 32, 4)
    B, _ = inputs.lstsq_rhs(A, 1, 1e-6, 6)
    Xo = oracle.lstsq(A, B)
    X0 = to_host(ts.lstsq(to_dev(A), to_dev(B), leaf_h=512, prec=ts.MIXED, max_refine=0))
    assert rel(X0, Xo) > 1e-8
    X64 = to_host(ts.lstsq(to_dev(A), to_dev(B), leaf_h=256, prec=ts.FP64))
    assert rel(X64, Xo) <= TOL


def test_mixed_singular(cuda_lib):
    import paper_0912_2572_gb300 as ts
    A = inputs.gaussian(2000, 6, 8)
    A[:, 2] = 0.0
    b = inputs.gaussian(2000, 1, 9)
    with pytest.raises(ts.TSQRError) as e:
        ts.lstsq(to_dev(A), to_dev(b), leaf_h=256, prec=ts.MIXED)
    assert e.value.status == 4


@pytest.mark.slow
def test_mixed_full_size_16M_by_32(cuda_lib):
    """The benchmark's mixed-precision workload: 16,777,216 x 32, sigma 1..1e-4, k = 4,
    b = A x_true + 1e-6 N(0,1)."""
    import paper_0912_2572_gb300 as ts
    m, n = 16_777_216, 32
    A = inputs.graded(m, n, 4.0, seed_g=0, seed_v=1)
    B, _ = inputs.lstsq_rhs(A, 4, 1e-6, 2)
    X, hist = ts.lstsq(to_dev(A), to_dev(B), leaf_h=512, arity=2, two_level=True, prec=ts.MIXED, max_refine=10,
                       info=True)
    Xo = oracle.lstsq(A, B)
    assert rel(to_host(X), Xo) <= TOL


def test_mixed_strided_and_many_rhs(cuda_lib):
    """lda > m, ldb > m, ldx > n, and k = 20 right-hand sides (three refinement groups)."""
    import torch
    import paper_0912_2572_gb300 as ts
    m, n, k = 30_000, 40, 20
    A = inputs.graded(m, n, 4.0, seed_g=3, seed_v=4)
    B, _ = inputs.lstsq_rhs(A, k, 1e-6, 5)
    Abig = torch.zeros((n, m + 11), dtype=torch.float64, device="cuda")
    Abig[:, :m] = torch.from_numpy(np.ascontiguousarray(A.T))
    Bbig = torch.zeros((k, m + 3), dtype=torch.float64, device="cuda")
    Bbig[:, :m] = torch.from_numpy(np.ascontiguousarray(B.T))
    Xbig = torch.full((k, n + 6), 5.0, dtype=torch.float64, device="cuda")
    X = Xbig.t()[:n]
    ts.lstsq(Abig.t()[:m], Bbig.t()[:m], prec=ts.MIXED, X=X)
    assert rel(to_host(X), oracle.lstsq(A, B)) <= TOL
    assert torch.all(Xbig[:, n:] == 5.0)


@pytest.mark.parametrize("m,n,dec,seed", [(20_000, 16, 4, 1), (50_000, 64, 3, 2), (8_000, 128, 2, 3)])
def test_gpu_refinement_against_oracle_csne(cuda_lib, m, n, dec, seed):
    """The GPU's refinement is corrected semi-normal equations iterated from x = 0 (Bjorck
    1987); the oracle runs the same iteration around its own FP32 Householder R. Both
    must land on the FP64 least-squares solution: the GPU x within 1e-10 of the oracle's
    CSNE x, each step's correction of the GPU history after the first smaller than the
    one before until the stop, and the first correction all of x (ratio 1)."""
    import paper_0912_2572_gb300 as ts
    A = inputs.graded(m, n, dec, seed_g=40 + seed, seed_v=50 + seed)
    b, _ = inputs.lstsq_rhs(A, 1, 1e-6, 60 + seed)
    X, hist = ts.lstsq(to_dev(A), to_dev(b), prec=ts.MIXED, max_refine=10, info=True)
    xg = to_host(X)[:, 0]
    xc, hc = oracle.lstsq_refine_csne(A, b[:, 0], max_steps=20, tol=1e-10)
    xo = oracle.lstsq(A, b[:, 0])
    assert rel(xc, xo) <= TOL
    assert rel(xg, xc) <= 2 * TOL
    h = [v for v in hist if v > 0]
    assert h[0] == 1.0 and 2 <= len(h) <= 6
    assert all(h[s + 1] < h[s] for s in range(len(h) - 1))
