"""The compact-WY FP32 leaf of the mixed path (tsqr_set_mixed_wy_min_n): chains factored
in 16-column panels whose reflectors update the trailing columns at once as I - V T V^T
(paper §2.2, the blocked Householder update), with V^T C and V (T^T W) on the tensor cores
as 3xTF32. R must match the oracle to FP32 leaf accuracy (as the unblocked FP32 chains),
the refined least-squares solutions must reach 1e-10 from the FP64 oracle, and an item
solved alone must be bitwise the same item inside a batch."""
import numpy as np
import pytest

import oracle
from paper_0912_2572_gb300 import inputs
from conftest import to_dev, to_host

pytestmark = pytest.mark.gpu


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.fixture
def wy_on(cuda_lib):
    import paper_0912_2572_gb300 as ts
    prev = ts.set_mixed_wy_min_n(17)
    yield
    ts.set_mixed_wy_min_n(prev)


# (m, n, k): one tile, several tiles per chain, ragged tails, every panel count
CASES = [(100, 32, 2), (3000, 48, 1), (20_000, 64, 4), (50_000, 100, 3), (130_000, 128, 2), (777, 128, 0),
         (40_000, 33, 8)]


@pytest.mark.parametrize("m,n,k", CASES)
def test_wy_leaf_matches_oracle(wy_on, m, n, k):
    import paper_0912_2572_gb300 as ts
    A = inputs.graded(m, n, 4.0, seed_g=m % 101, seed_v=n)
    item = {"A": to_dev(A), "prec": ts.MIXED}
    if k:
        B, _ = inputs.lstsq_rhs(A, k, 1e-6, 3)
        item["B"] = to_dev(B)
    outs, st, info = ts.batch_solve([item], chain_tiles=4, status=True, info=True)
    assert st == [0]
    R, X = outs[0]
    R = to_host(R)
    assert np.all(np.diag(R) >= 0) and np.all(np.tril(R, -1) == 0)
    assert rel(R, oracle.r_factor(A)) <= 1e-5
    prev = ts.set_mixed_wy_min_n(0)  # the unblocked FP32 chains on the same item
    outs0, info0 = ts.batch_solve([item], chain_tiles=4, info=True)
    ts.set_mixed_wy_min_n(prev)
    Ro = oracle.r_factor(A)
    print(f"m={m} n={n} k={k}: R err wy {rel(R, Ro):.2e} unblocked {rel(to_host(outs0[0][0]), Ro):.2e}; "
          f"refinement steps wy {info[0][0]} unblocked {info0[0][0]}")
    if k:
        assert rel(to_host(X), oracle.lstsq(A, B)) <= 1e-10
        assert info[0][0] <= 10


def test_wy_leaf_agrees_with_unblocked_chains(cuda_lib):
    """The blocked and the unblocked FP32 chains compute the same R up to FP32 rounding."""
    import paper_0912_2572_gb300 as ts
    A = inputs.gaussian(30_000, 96, 11)
    Rs = []
    for thr in (0, 17):
        prev = ts.set_mixed_wy_min_n(thr)
        (R, _), = ts.batch_solve([{"A": to_dev(A), "prec": ts.MIXED}], chain_tiles=8)
        ts.set_mixed_wy_min_n(prev)
        Rs.append(to_host(R))
    assert rel(Rs[1], Rs[0]) <= 2e-6


def test_wy_alone_equals_in_mix(wy_on):
    import paper_0912_2572_gb300 as ts
    items, host = [], []
    for q in range(8):
        n = (24, 40, 64, 128)[q % 4]
        m = 2000 + 7000 * q
        A = inputs.graded(m, n, 3.0, seed_g=q, seed_v=q + 9)
        B, _ = inputs.lstsq_rhs(A, 2, 1e-6, q + 20)
        items.append({"A": to_dev(A), "B": to_dev(B), "prec": ts.MIXED if q % 3 else ts.FP64})
        host.append((A, B))
    mix = ts.batch_solve(items, chain_tiles=8)
    for q in (1, 2, 7):
        (R1, X1), = ts.batch_solve([items[q]], chain_tiles=8)
        assert np.array_equal(to_host(R1), to_host(mix[q][0]))
        assert np.array_equal(to_host(X1), to_host(mix[q][1]))
        assert rel(to_host(X1), oracle.lstsq(*host[q])) <= 1e-10
