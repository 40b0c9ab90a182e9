"""The tile-pair kernel for one right-hand side (Q^T b and Q b, paper §2.3: the implicit Q
applied tile by tile along each flat chain and tree node). A job's tiles alternate between
the two half-warps of its warp, one reflector step apart. Checked against the oracle's
Q^T b (the unique top n entries and the norm of the rest) and Q c, against the one-warp-
per-tile kernel (the same products in another summation order), and by the round trip
Q (Q^T b) = b, over plans whose jobs hold one, two, an odd and an even number of tiles,
ragged last tiles, the tree's triangle pieces, a flat tree of one job and n = 2, the
smallest width the pair schedule takes (n = 1 keeps the warp kernel)."""
import numpy as np
import pytest

import oracle
from paper_0912_2572_gb300 import inputs
from conftest import to_dev, to_host

pytestmark = pytest.mark.gpu


def rel(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / (nb if nb > 0 else 1.0)


# (m, n, leaf_h, arity, two_level)
SHAPES = [
    (20_000, 2, 1000, 2, False),      # n = 2; leaves of several tiles
    (30_011, 16, 1000, 4, False),     # ragged leaves; 4-ary tree levels (3 tiles per job)
    (9_001, 7, 50, 0, False),         # flat tree: one job of every tile
    (2_000_003, 32, 144, 2, True),    # two-level chains of 7-8 tiles, ragged counts
    (700, 100, 150, 3, True),         # n = 100: tree triangles in pieces
    (100_000, 128, 512, 2, False),    # the tallest tiles the plan makes at n = 128
    (1_000, 1, 64, 2, False),         # n = 1: the warp kernel
]


def _apply_both(F, b, trans):
    import paper_0912_2572_gb300 as ts
    out = {}
    for pairs in (False, True):
        prev = ts.set_apply_tile_pairs(pairs)
        try:
            bd = to_dev(b)
            (F.apply_qt if trans else F.apply_q)(bd)
            out[pairs] = to_host(bd)
        finally:
            ts.set_apply_tile_pairs(prev)
    return out[False], out[True]


@pytest.mark.parametrize("m,n,h,arity,two", SHAPES)
def test_tile_pairs_qt_b(cuda_lib, m, n, h, arity, two):
    import paper_0912_2572_gb300 as ts
    A = inputs.gaussian(m, n, seed=m % 997 + n)
    b = inputs.gaussian(m, 1, seed=n + 1000)
    F = ts.factor(to_dev(A), leaf_h=h, arity=arity, two_level=two)
    warp, pairs = _apply_both(F, b, trans=True)
    if m <= 100_000:
        top, tail = oracle.qt_b(A, b)
        assert rel(pairs[:n], top) <= 1e-12
        assert rel(np.linalg.norm(pairs[n:], axis=0), tail) <= 1e-12
    assert rel(pairs, warp) <= 1e-13
    # Q (Q^T b) = b through the pair kernel
    bd = to_dev(pairs)
    F.apply_q(bd)
    assert rel(to_host(bd), b) <= 1e-13
    F.free()


@pytest.mark.parametrize("m,n,h,arity,two", SHAPES)
def test_tile_pairs_q_c(cuda_lib, m, n, h, arity, two):
    """Q [c; 0] for coordinates c: the thin Q times c, against the oracle's Q."""
    import paper_0912_2572_gb300 as ts
    A = inputs.gaussian(m, n, seed=m % 991 + 2 * n)
    c = inputs.gaussian(n, 1, seed=n + 7)
    F = ts.factor(to_dev(A), leaf_h=h, arity=arity, two_level=two)
    b = np.zeros((m, 1))
    b[:n] = c
    warp, pairs = _apply_both(F, b, trans=False)
    assert rel(pairs, warp) <= 1e-13
    if m <= 100_000:
        Qo, _, _ = oracle.qr(A)
        assert rel(pairs, Qo @ c) <= 1e-12
    F.free()


def test_tile_pairs_full_chain(cuda_lib):
    """At 4,194,304 x 64 (1,824 chains of 16 tiles): Q^T b by tile pairs equals the one-warp
    kernel's to rounding and keeps the norm of b; its top n entries are R x for the least-
    squares x (tsqr_lstsq factors [A | b], so that x comes without this kernel); and the
    Q^T b overlapped with the factorization is bitwise that of tsqr_apply_qt afterwards."""
    import torch
    import paper_0912_2572_gb300 as ts
    m, n = 1 << 22, 64
    A = inputs.gaussian(m, n, seed=31)
    b = inputs.gaussian(m, 1, seed=33)
    Ad, bd = to_dev(A), to_dev(b)
    F = ts.factor(Ad, leaf_h=144, two_level=True)
    warp, pairs = _apply_both(F, b, trans=True)
    assert rel(pairs, warp) <= 1e-13
    assert abs(np.linalg.norm(pairs) - np.linalg.norm(b)) <= 1e-13 * np.linalg.norm(b)
    x = to_host(ts.lstsq(Ad, bd, leaf_h=144))
    assert rel(to_host(F.R) @ x, pairs[:n]) <= 1e-12
    q2 = to_dev(b)
    F2 = ts.factor(Ad, leaf_h=144, two_level=True, qt=q2)
    assert np.array_equal(to_host(q2), pairs)
    F.free()
    F2.free()
    torch.cuda.synchronize()
    assert ts.error_word() == 0
