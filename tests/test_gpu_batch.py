"""The persistent batched engine: many uneven problems in one launch (chain jobs from a
device queue; the last child to arrive at a tree node runs its combine, paper §2.3).
Each item must match the oracle, and be bitwise identical alone and inside a batch."""
import numpy as np
import pytest

import oracle
from paper_0912_2572_gb300 import inputs
from conftest import to_dev, to_host

pytestmark = pytest.mark.gpu


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def make_items(count, seed, mlo=256, mhi=20000, ns=(8, 16, 32, 64), mixed_share=0.5, k=0):
    g = inputs.rng(seed)
    out = []
    for q in range(count):
        m = int(np.exp(g.uniform(np.log(mlo), np.log(mhi))))
        n = int(g.choice(ns))
        m = max(m, n)
        A = inputs.gaussian(m, n, seed * 1000 + q)
        prec = 1 if (k == 0 and g.uniform() < mixed_share) else 0
        B = inputs.gaussian(m, k, seed * 1000 + q + 500) if k else None
        out.append((A, B, prec))
    return out


def run(items, **kw):
    import paper_0912_2572_gb300 as ts
    dev = [{"A": to_dev(A), "prec": p, **({"B": to_dev(B)} if B is not None else {})} for A, B, p in items]
    outs, st = ts.batch_solve(dev, status=True, **kw)
    return [(to_host(R), to_host(X) if X is not None else None) for R, X in outs], st


def test_batch_factor_matches_oracle(cuda_lib):
    items = make_items(60, 1)
    res, st = run(items)
    assert st == [0] * len(items)
    for (A, _, prec), (R, _) in zip(items, res):
        Ro = oracle.r_factor(A)
        assert np.all(np.diag(R) >= 0) and np.all(np.tril(R, -1) == 0)
        # FP64 items to 1e-12; FP32-mixed items carry single-precision leaf rounding
        assert rel(R, Ro) <= (1e-12 if prec == 0 else 1e-5)


def test_batch_alone_equals_in_mix(cuda_lib):
    items = make_items(40, 2)
    res_mix, _ = run(items)
    for q in (0, 7, 23, 39):
        res_alone, _ = run([items[q]])
        assert np.array_equal(res_alone[0][0], res_mix[q][0])


def test_batch_least_squares(cuda_lib):
    items = make_items(30, 3, k=3, ns=(16, 32, 64, 100))
    res, st = run(items)
    assert st == [0] * len(items)
    for (A, B, _), (R, X) in zip(items, res):
        assert rel(X, oracle.lstsq(A, B)) <= 1e-12
        assert rel(R, oracle.r_factor(A)) <= 1e-12


def test_batch_tree_shapes_and_chain_lengths(cuda_lib):
    items = make_items(12, 4, mlo=5000, mhi=60000)
    ref, _ = run(items, chain_tiles=8, arity=2)
    for ct, ar in ((1, 2), (3, 4), (64, 16)):
        res, _ = run(items, chain_tiles=ct, arity=ar)
        for (A, _, prec), (R, _), (R0, _) in zip(items, res, ref):
            assert rel(R, R0) <= (1e-12 if prec == 0 else 1e-5)


def test_batch_singular_item(cuda_lib):
    A = inputs.gaussian(3000, 8, 9)
    A[:, 5] = 0.0
    B = inputs.gaussian(3000, 1, 10)
    good = make_items(3, 5, k=1)
    res, st = run([good[0], (A, B, 0), good[1]])
    assert st == [0, 4, 0]
    assert rel(res[0][1], oracle.lstsq(good[0][0], good[0][1])) <= 1e-12


@pytest.mark.parametrize("n,k", [(128, 8), (128, 16), (120, 20), (100, 3)])
def test_batch_wide_least_squares(cuda_lib, n, k):
    """n + k up to 144: the persistent kernel's ninth column slot per half-warp."""
    g = inputs.rng(n * 100 + k)
    items = []
    for q in range(5):
        m = int(g.integers(n, 30000))
        A = inputs.graded(m, n, 3.0, seed_g=q + 40, seed_v=q + 41)
        B, _ = inputs.lstsq_rhs(A, k, 1e-6, q + 42)
        items.append((A, B, 0))
    res, st = run(items, chain_tiles=4)
    assert st == [0] * len(items)
    for (A, B, _), (R, X) in zip(items, res):
        assert rel(R, oracle.r_factor(A)) <= 1e-12
        assert rel(X, oracle.lstsq(A, B)) <= 1e-10


def lsq_items(count, seed, prec, ns=(16, 32, 64, 100, 128), kmax=12, mhi=40000, dec_max=4.0):
    g = inputs.rng(seed)
    out = []
    for q in range(count):
        n = int(g.choice(ns))
        m = max(int(np.exp(g.uniform(np.log(300), np.log(mhi)))), n)
        k = int(g.integers(1, kmax + 1))
        A = inputs.graded(m, n, float(g.uniform(0.0, dec_max)), seed_g=seed * 1000 + q, seed_v=seed * 1000 + q + 1)
        B, _ = inputs.lstsq_rhs(A, k, 1e-6, seed * 1000 + q + 2)
        out.append((A, B, prec))
    return out


def test_batch_mixed_least_squares_matches_oracle(cuda_lib):
    """FP32 leaf chains, FP64 tree, FP64 refinement by corrected semi-normal equations:
    ||x - x_oracle|| / ||x_oracle|| <= 1e-10 for kappa <= 1e4, including k > 8 (two
    refinement groups) and ragged row blocks."""
    items = lsq_items(24, 11, prec=1)
    res, st = run(items)
    assert st == [0] * len(items)
    for (A, B, _), (R, X) in zip(items, res):
        assert rel(X, oracle.lstsq(A, B)) <= 1e-10
        assert rel(R, oracle.r_factor(A)) <= 1e-5  # R itself carries the FP32 leaves


def test_batch_mixed_refinement_needs_more_than_one_step(cuda_lib):
    """kappa = 1e4: the first semi-normal solve alone is far from FP64 accuracy, so the
    result above is the refinement's doing."""
    import paper_0912_2572_gb300 as ts
    A = inputs.graded(20000, 64, 4.0, seed_g=5, seed_v=6)
    B, _ = inputs.lstsq_rhs(A, 2, 1e-6, 7)
    Xo = oracle.lstsq(A, B)
    (R, X), = ts.batch_solve([{"A": to_dev(A), "B": to_dev(B), "prec": ts.MIXED}])
    assert rel(to_host(X), Xo) <= 1e-10
    # a plain FP32-accurate solve with the same R: x1 = R^{-1} R^{-T} A^T b
    Rh = to_host(R)
    x1 = np.linalg.solve(Rh, np.linalg.solve(Rh.T, A.T @ B))
    assert rel(x1, Xo) > 1e-8


def test_batch_auto_and_mixed_alone_equals_in_mix(cuda_lib):
    items = lsq_items(16, 12, prec=2, kmax=8) + lsq_items(8, 13, prec=1, kmax=10)
    res_mix, st = run(items, chain_tiles=8)
    assert st == [0] * len(items)
    for q in (0, 5, 17, 23):
        res_alone, _ = run([items[q]], chain_tiles=8)
        assert np.array_equal(res_alone[0][1], res_mix[q][1])
        assert np.array_equal(res_alone[0][0], res_mix[q][0])
    for (A, B, _), (R, X) in zip(items, res_mix):
        assert rel(X, oracle.lstsq(A, B)) <= 1e-10


def test_batch_mixed_singular_item(cuda_lib):
    A = inputs.gaussian(5000, 12, 19)
    A[:, 3] = 0.0
    B = inputs.gaussian(5000, 2, 20)
    good = lsq_items(2, 14, prec=1, kmax=3)
    _, st = run([good[0], (A, B, 1), good[1]])
    assert st == [0, 4, 0]


def test_batch_plan_replay_equals_batch_solve(cuda_lib):
    """A plan captured once as a CUDA graph gives bitwise the results of tsqr_batch_solve,
    and picks up new data written in place into the same buffers."""
    import torch
    import paper_0912_2572_gb300 as ts
    items = lsq_items(10, 21, prec=2, kmax=9) + make_items(6, 22)
    dev = [{"A": to_dev(A), "prec": p, **({"B": to_dev(B)} if B is not None else {})} for A, B, p in items]
    ref, st = ts.batch_solve(dev, chain_tiles=8, status=True)
    with ts.BatchPlan(dev, chain_tiles=8) as plan:
        for _ in range(2):
            outs = plan.run()
            status, info = plan.results()
            assert status == st
            for (R0, X0), (R1, X1) in zip(ref, outs):
                assert torch.equal(R0, R1)
                if X0 is not None:
                    assert torch.equal(X0, X1)
        # new data in the same buffers
        for q, d in enumerate(dev):
            d["A"].mul_(2.0)
        outs = plan.run()
        plan.results()
        ref2 = ts.batch_solve(dev, chain_tiles=8)
        for (R0, X0), (R1, X1) in zip(ref2, outs):
            assert torch.equal(R0, R1)
            if X0 is not None:
                assert torch.equal(X0, X1)
        for (A, B, p), (R, X) in zip(items[:10], outs[:10]):
            # A doubled: x halves
            assert rel(to_host(X) * 2.0, oracle.lstsq(A, B)) <= 1e-10


def test_batch_strided_layouts(cuda_lib):
    """Leading dimensions larger than the rows (views into bigger arrays) for A, B, R and X,
    FP64 and mixed items alike."""
    import torch
    import paper_0912_2572_gb300 as ts
    g = inputs.rng(31)
    items, host = [], []
    for q, prec in enumerate((ts.FP64, ts.MIXED, ts.AUTO, ts.FP64)):
        m, n, k = int(g.integers(500, 9000)), int(g.choice([8, 32, 60])), int(g.integers(1, 6))
        A = inputs.graded(m, n, 3.0, seed_g=100 + q, seed_v=200 + q)
        B, _ = inputs.lstsq_rhs(A, k, 1e-6, 300 + q)
        Abig = torch.zeros((n, m + 37), dtype=torch.float64, device="cuda")
        Abig[:, :m] = torch.from_numpy(np.ascontiguousarray(A.T))
        Bbig = torch.zeros((k, m + 5), dtype=torch.float64, device="cuda")
        Bbig[:, :m] = torch.from_numpy(np.ascontiguousarray(B.T))
        Rbig = torch.full((n, n + 3), 7.0, dtype=torch.float64, device="cuda")
        Xbig = torch.full((k, n + 9), 7.0, dtype=torch.float64, device="cuda")
        items.append({"A": Abig.t()[:m], "B": Bbig.t()[:m], "R": Rbig.t()[:n], "X": Xbig.t()[:n], "prec": prec})
        host.append((A, B, prec, Rbig, Xbig))
    outs, st = ts.batch_solve(items, status=True)
    assert st == [0] * len(items)
    for (A, B, prec, Rbig, Xbig), (R, X) in zip(host, outs):
        n = A.shape[1]
        assert rel(to_host(X), oracle.lstsq(A, B)) <= 1e-10
        assert rel(to_host(R), oracle.r_factor(A)) <= (1e-12 if prec == ts.FP64 else 1e-5)
        # padding past the leading rows is untouched
        assert torch.all(Rbig[:, n:] == 7.0) and torch.all(Xbig[:, n:] == 7.0)


@pytest.mark.parametrize("m,n,k,prec", [(1, 1, 1, 0), (1, 1, 1, 1), (7, 1, 3, 1), (128, 128, 0, 0), (128, 128, 0, 1),
                                        (129, 128, 8, 1), (128, 120, 8, 0), (16, 16, 1, 1), (5000, 1, 0, 1),
                                        (300, 64, 0, 2)])
def test_batch_degenerate_shapes(cuda_lib, m, n, k, prec):
    """Single-row and single-column problems, m = n (one tile, no tree), R-only mixed
    items, k = 0 FP64 items; alone and next to an ordinary item."""
    A = inputs.graded(m, n, 2.0, seed_g=m + n, seed_v=k + 3) if n > 1 else inputs.gaussian(m, n, m)
    B = inputs.gaussian(m, k, m + 1) if k else None
    other = make_items(1, 40, k=0)[0]
    res, st = run([(A, B, prec), other])
    assert st == [0, 0]
    R, X = res[0]
    tolr = 1e-12 if prec in (0, 2) else 1e-5
    assert rel(R, oracle.r_factor(A)) <= tolr
    if k:
        assert rel(X, oracle.lstsq(A, B)) <= 1e-10


def test_batch_of_ten_thousand_sampled_against_oracle(cuda_lib):
    """The batched workload at full size: 10,000 instances, m log-uniform in [256, 65,536],
    n from {8, 16, 32, 64}, iid N(0,1) from a seeded device generator, alternately FP64 and
    FP32-mixed, in one launch (chain length 16, binary tree). A seeded sample of 100 items
    is checked against the oracle (FP64 items to 1e-12, mixed R-only items to FP32 leaf
    accuracy, 1e-5), and every item's status is 0."""
    import torch
    import paper_0912_2572_gb300 as ts
    count = 10_000
    g = inputs.rng(17)
    ms = np.exp(g.uniform(np.log(256), np.log(65536), size=count)).astype(np.int64)
    ns = g.choice([8, 16, 32, 64], size=count)
    ms = np.maximum(ms, ns)
    offs = np.concatenate([[0], np.cumsum(ms * ns)])
    gen = torch.Generator(device="cuda")
    gen.manual_seed(17)
    buf = torch.randn(int(offs[-1]), dtype=torch.float64, device="cuda", generator=gen)
    items = [{"A": buf[offs[q]:offs[q + 1]].view(int(ns[q]), int(ms[q])).t(), "prec": q & 1} for q in range(count)]
    outs, st = ts.batch_solve(items, chain_tiles=16, arity=2, status=True)
    assert st == [0] * count
    sample = inputs.rng(18).choice(count, size=100, replace=False)
    for q in sample:
        A = to_host(items[q]["A"])
        R = to_host(outs[q][0])
        assert np.all(np.diag(R) >= 0) and np.all(np.tril(R, -1) == 0)
        assert rel(R, oracle.r_factor(A)) <= (1e-12 if q % 2 == 0 else 1e-5), f"item {q}"
    del buf, items, outs
    torch.cuda.empty_cache()
