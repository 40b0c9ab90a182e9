"""The cluster tier of the reduction tree (TSQR_CLUSTER; paper §2.3 and §3, the
hierarchical tree: CTA chains, then combines inside thread-block clusters that exchange
their triangles through distributed shared memory, then the grid). It runs the same
combine jobs with the same arithmetic as the per-level binary tree, so R, the thin Q and
Q^T b are bitwise those of the binary tree, and R matches the oracle. The device error
word must stay clear (no bounded wait gave up)."""
import numpy as np
import pytest

import oracle
from paper_0912_2572_gb300 import inputs
from conftest import to_dev, to_host

pytestmark = pytest.mark.gpu


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


CASES = [
    # (m, n, leaf_h, two_level): 16 leaves (2 cluster launches), 1,562 leaves (11 levels),
    # leaf counts that leave lone nodes and partial clusters, a 3-leaf tree, the headline's
    # two-level shape at 1M rows, and a width that is not a multiple of 8
    (4096, 16, 256, False),
    (100_000, 32, 64, False),
    (5000, 64, 64, False),
    (3000, 16, 100, False),
    (640, 64, 64, False),
    (200, 8, 64, False),
    (1 << 20, 64, 144, True),
    (300_000, 37, 144, True),
]


@pytest.mark.parametrize("m,n,h,two", CASES)
def test_cluster_tree_bitwise_and_oracle(cuda_lib, m, n, h, two):
    import paper_0912_2572_gb300 as ts
    A = inputs.graded(m, n, 6.0, seed_g=m % 1000 + n, seed_v=7) if m >= 100_000 else inputs.gaussian(m, n, m + n)
    Ad = to_dev(A)
    out = {}
    for cl in (False, True):
        F = ts.factor(Ad, leaf_h=h, arity=2, two_level=two, cluster=cl)
        Q = F.form_q()
        b = to_dev(inputs.gaussian(m, 2, 5))
        F.apply_qt(b)
        out[cl] = (to_host(F.R), to_host(Q), to_host(b), F.info())
        F.free()
    assert ts.error_word() == 0
    R0, Q0, b0, i0 = out[False]
    R1, Q1, b1, i1 = out[True]
    assert np.array_equal(R1, R0) and np.array_equal(Q1, Q0) and np.array_equal(b1, b0)
    if i0["launches"] > 3:
        assert i1["launches"] < i0["launches"]
    assert _rel(R1, oracle.r_factor(A)) <= 1e-12
    if m <= 100_000:
        assert oracle.orth_error(Q1) <= 1e-13
    else:  # the oracle's O(m n^2) compensated sums are slow here: orthogonality by a product
        assert np.linalg.norm(Q1.T @ Q1 - np.eye(n)) <= 1e-13


def test_cluster_tree_least_squares_and_caqr(cuda_lib):
    """The fused least-squares factorization (n + k columns through the tree) and CAQR's
    panels with the cluster tier: bitwise equal to the binary tree, and the oracle."""
    import paper_0912_2572_gb300 as ts
    m, n, k = 50_000, 48, 3
    A = inputs.graded(m, n, 3.0, seed_g=81, seed_v=82)
    B, _ = inputs.lstsq_rhs(A, k, 1e-4, 83)
    X0 = to_host(ts.lstsq(to_dev(A), to_dev(B), leaf_h=128, two_level=False))
    X1 = to_host(ts.lstsq(to_dev(A), to_dev(B), leaf_h=128, two_level=False, cluster=True))
    assert np.array_equal(X1, X0)
    assert _rel(X1, oracle.lstsq(A, B)) <= 1e-12
    Aw = inputs.gaussian(20_000, 160, 84)
    F0 = ts.caqr(to_dev(Aw), leaf_h=144)
    F1 = ts.caqr(to_dev(Aw), leaf_h=144, cluster=True)
    assert np.array_equal(to_host(F1.R), to_host(F0.R))
    assert np.array_equal(to_host(F1.form_q()), to_host(F0.form_q()))
    F0.free()
    F1.free()
    assert ts.error_word() == 0


def test_cluster_tree_overlapped_apply(cuda_lib):
    """tsqr_factor_qt pairs each Q^T B tree level with the factorization launch that
    completes it; with cluster launches a launch completes three levels."""
    import paper_0912_2572_gb300 as ts
    m, n = 200_000, 32
    A = inputs.gaussian(m, n, 85)
    B = inputs.gaussian(m, 4, 86)
    Ad = to_dev(A)
    ref = to_dev(B)
    F0 = ts.factor(Ad, leaf_h=64, arity=2, two_level=False)
    F0.apply_qt(ref)
    qb = to_dev(B)
    F1 = ts.factor(Ad, leaf_h=64, arity=2, two_level=False, cluster=True, qt=qb)
    assert np.array_equal(to_host(qb), to_host(ref))
    assert np.array_equal(to_host(F1.R), to_host(F0.R))
    F0.free()
    F1.free()


@pytest.mark.parametrize("m,n,k", [(1 << 20, 64, 0), (300_000, 48, 0), (200_000, 32, 24), (60_000, 100, 12)])
def test_cluster_apply_top_down_bitwise(cuda_lib, m, n, k):
    """The thin Q (k = 0) and Q B (k > 8 columns) through the cluster tier of the apply (the
    tree levels run top down in clusters, pipelined through distributed shared memory) are
    bitwise those of the per-level launches; Q^T (Q B) = B and the thin Q is orthonormal."""
    import torch
    import paper_0912_2572_gb300 as ts
    A = inputs.gaussian(m, n, m % 1000 + n)
    Ad = to_dev(A)
    F0 = ts.factor(Ad, leaf_h=144, two_level=True)
    F1 = ts.factor(Ad, leaf_h=144, two_level=True, cluster=True)
    if k == 0:
        Q0, Q1 = to_host(F0.form_q()), to_host(F1.form_q())
        assert np.array_equal(Q1, Q0)
        assert np.linalg.norm(Q1.T @ Q1 - np.eye(n)) <= 1e-13
    else:
        B = inputs.gaussian(m, k, 7)
        B0, B1 = to_dev(B), to_dev(B)
        F0.apply_q(B0)
        F1.apply_q(B1)
        assert np.array_equal(to_host(B1), to_host(B0))
        F1.apply_qt(B1)
        assert _rel(to_host(B1), B) <= 1e-13
    F0.free()
    F1.free()
    torch.cuda.synchronize()
    assert ts.error_word() == 0
