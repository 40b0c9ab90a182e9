"""GPU parity of the implicit Q (paper §4, Table 2): Q^T B, Q B, least squares through
Q^T b and back substitution, in-place factorization, singular input, and the
tree-shape independence of paper §2.3 (associativity of the reduce operator)."""
import numpy as np
import pytest

import oracle
from paper_0912_2572_gb300 import inputs
from conftest import to_dev, to_host

pytestmark = pytest.mark.gpu


def rel(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / (nb if nb > 0 else 1.0)


SHAPES = [
    (4096, 16, 256, 2, False),
    (5000, 64, 216, 2, True),
    (3001, 32, 100, 4, False),
    (2000, 8, 300, 0, False),
    (700, 100, 150, 3, True),
]


@pytest.mark.parametrize("m,n,h,arity,two", SHAPES)
@pytest.mark.parametrize("k", [1, 3, 8, 17, 70])
def test_apply_qt_unique_part(cuda_lib, m, n, h, arity, two, k):
    import paper_0912_2572_gb300 as ts
    A = inputs.gaussian(m, n, seed=1)
    B = inputs.gaussian(m, k, seed=2)
    F = ts.factor(to_dev(A), leaf_h=h, arity=arity, two_level=two)
    Bd = to_dev(B)
    F.apply_qt(Bd)
    C = to_host(Bd)
    top, tail = oracle.qt_b(A, B)
    assert rel(C[:n], top) <= 1e-12
    assert rel(np.linalg.norm(C[n:], axis=0), tail) <= 1e-12
    # Q (Q^T B) = B
    F.apply_q(Bd)
    assert rel(to_host(Bd), B) <= 1e-13
    F.free()


@pytest.mark.parametrize("m,n,h,arity,two,k", [(300_011, 64, 144, 2, True, 1), (50_003, 32, 100, 4, False, 12),
                                               (20_000, 16, 256, 0, False, 3), (9_001, 7, 50, 3, True, 70)])
def test_factor_qt_equals_factor_then_apply(cuda_lib, m, n, h, arity, two, k):
    """tsqr_factor_qt overlaps Q^T B with the factorization's tree on a helper stream; its
    R, B and factor set are bitwise those of tsqr_factor + tsqr_apply_qt."""
    import paper_0912_2572_gb300 as ts
    A = inputs.gaussian(m, n, 51)
    B = inputs.gaussian(m, k, 52)
    Ad = to_dev(A)
    B1 = to_dev(B)
    F1 = ts.factor(Ad, leaf_h=h, arity=arity, two_level=two)
    F1.apply_qt(B1)
    B2 = to_dev(B)
    F2 = ts.factor(Ad, leaf_h=h, arity=arity, two_level=two, qt=B2)
    assert np.array_equal(to_host(F2.R), to_host(F1.R))
    assert np.array_equal(to_host(B2), to_host(B1))
    top, _ = oracle.qt_b(A, B)
    assert rel(to_host(B2)[:n], top) <= 1e-12
    assert np.array_equal(to_host(F2.form_q()), to_host(F1.form_q()))
    F1.free()
    F2.free()


@pytest.mark.parametrize("m,n,h,two", [(200_003, 16, 64, False), (131_077, 8, 32, True)])
def test_apply_one_rhs_over_many_jobs(cuda_lib, m, n, h, two):
    """A single right-hand side over a chain launch of thousands of jobs (one warp per job),
    with the remainder rows in the last leaf, so the jobs differ in tile count and height."""
    import paper_0912_2572_gb300 as ts
    info = ts.plan_describe(m, n, h, 2, two)
    assert info["jobs"] >= 1024
    A = inputs.gaussian(m, n, seed=13)
    b = inputs.gaussian(m, 1, seed=14)
    F = ts.factor(to_dev(A), leaf_h=h, arity=2, two_level=two)
    bd = to_dev(b)
    F.apply_qt(bd)
    c = to_host(bd)
    top, tail = oracle.qt_b(A, b)
    assert rel(c[:n], top) <= 1e-12
    assert rel(np.linalg.norm(c[n:], axis=0), tail) <= 1e-12
    F.apply_q(bd)
    assert rel(to_host(bd), b) <= 1e-13
    F.free()


@pytest.mark.parametrize("m,n,h,arity,two", SHAPES)
def test_apply_q_of_thin_coordinates(cuda_lib, m, n, h, arity, two):
    """Q [c; 0] = Q_thin c, the only part of Q B fixed by the factorization."""
    import paper_0912_2572_gb300 as ts
    A = inputs.gaussian(m, n, seed=3)
    c = inputs.gaussian(n, 2, seed=4)
    F = ts.factor(to_dev(A), leaf_h=h, arity=arity, two_level=two)
    Bc = np.zeros((m, 2))
    Bc[:n] = c
    Bd = to_dev(Bc)
    F.apply_q(Bd)
    Qo, _, _ = oracle.qr(A)
    assert rel(to_host(Bd), Qo @ c) <= 1e-12
    F.free()


@pytest.mark.parametrize("m,n,k,h,arity,two,dec", [
    (4096, 16, 1, 256, 2, False, 0), (5000, 64, 4, 216, 2, True, 4), (3000, 32, 8, 128, 4, False, 4),
    (2000, 100, 40, 200, 2, True, 2), (1500, 64, 64, 150, 0, False, 0), (257, 1, 2, 1, 2, False, 0)])
def test_lstsq_matches_oracle(cuda_lib, m, n, k, h, arity, two, dec):
    import paper_0912_2572_gb300 as ts
    A = inputs.graded(m, n, dec) if dec else inputs.gaussian(m, n, 5)
    B, _ = inputs.lstsq_rhs(A, k, 1e-3, 6)
    X = to_host(ts.lstsq(to_dev(A), to_dev(B), leaf_h=h, arity=arity, two_level=two))
    Xo = oracle.lstsq(A, B)
    tol = 1e-12 if dec <= 2 else 1e-10  # forward error grows with kappa = 10^dec
    assert rel(X, Xo) <= tol
    # the same through apply_qt + solve_r on a kept factor set
    F = ts.factor(to_dev(A), leaf_h=h, arity=arity, two_level=two)
    Cd = to_dev(B)
    F.apply_qt(Cd)
    X2 = to_host(F.solve_r(Cd))
    assert rel(X2, Xo) <= tol
    F.free()


def test_inplace_factor(cuda_lib):
    import paper_0912_2572_gb300 as ts
    A = inputs.gaussian(3000, 24, 7)
    Ad = to_dev(A)
    F = ts.factor(Ad, leaf_h=200, arity=2, two_level=True, inplace=True)
    Q = to_host(F.form_q())
    R = to_host(F.R)
    Qo, Ro, _ = oracle.qr(A)
    assert rel(R, Ro) <= 1e-12 and rel(Q, Qo) <= 1e-12
    assert not np.array_equal(to_host(Ad), A)  # reflectors overwrote A
    F.free()


def test_singular_least_squares(cuda_lib):
    import paper_0912_2572_gb300 as ts
    A = inputs.gaussian(1000, 6, 8)
    A[:, 3] = 0.0
    b = inputs.gaussian(1000, 1, 9)
    with pytest.raises(ts.TSQRError) as e:
        ts.lstsq(to_dev(A), to_dev(b), leaf_h=128, arity=2)
    assert e.value.status == 4
    # the factorization itself succeeds: r_33 = 0, backward error at rounding level
    F = ts.factor(to_dev(A), leaf_h=128, arity=2)
    R = to_host(F.R)
    Q = to_host(F.form_q())
    assert R[3, 3] == 0.0
    assert oracle.backward_error(A, Q, R) <= 1e-14
    F.free()


def test_tree_shapes_agree(cuda_lib):
    """Every tree shape and leaf height gives the same R (associativity, paper §2.3)."""
    import paper_0912_2572_gb300 as ts
    m, n = 65536, 48
    A = inputs.graded(m, n, 6)
    Ad = to_dev(A)
    Ro = oracle.r_factor(A)
    Rs = []
    for h, arity, two in [(64, 2, False), (128, 4, False), (256, 2, True), (1024, 0, True), (512, 3, False),
                          (1000, 0, False), (216, 16, True)]:
        F = ts.factor(Ad, leaf_h=h, arity=arity, two_level=two)
        Rs.append(to_host(F.R))
        F.free()
    for R in Rs:
        assert rel(R, Ro) <= 1e-12
        assert rel(R, Rs[0]) <= 1e-12


def test_edge_shapes(cuda_lib):
    """Square A, m = n + 1, one leaf, a ragged last tile, n = 1."""
    import paper_0912_2572_gb300 as ts
    for m, n, h, arity in [(128, 128, 128, 2), (65, 64, 64, 2), (100, 7, 100, 2), (217, 64, 216, 2),
                           (1, 1, 1, 2), (2, 1, 1, 2), (33, 1, 4, 3)]:
        A = inputs.gaussian(m, n, m + n)
        F = ts.factor(to_dev(A), leaf_h=h, arity=arity)
        Q = to_host(F.form_q())
        R = to_host(F.R)
        Qo, Ro, _ = oracle.qr(A)
        assert rel(R, Ro) <= 1e-12, (m, n)
        assert rel(Q, Qo) <= 1e-12, (m, n)
        F.free()
