"""Q-only TSQR (tsqr_orthonormalize): the orthogonalization step of block iterative
methods, the use of TSQR the paper names beside CAQR's panel (§2.5, §6). The basis must
match the oracle's thin Q (unique for full-rank A once diag(R) >= 0, §4 Property 1),
equal tsqr_factor + tsqr_form_q bitwise, and work in place."""
import numpy as np
import pytest

import oracle
from paper_0912_2572_gb300 import inputs
from conftest import to_dev, to_host

pytestmark = pytest.mark.gpu

R_TOL = 1e-12      # relative Frobenius error of R and Q against the oracle
BE_TOL = 1e-13     # ||A - QR||_F / ||A||_F and ||Q^T Q - I||_F


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


CASES = [
    (4096, 16, 256, 2, False),
    (50_003, 8, 100, 4, False),
    (9_001, 32, 64, 0, False),
    (300_011, 64, 144, 2, True),
    (1_000, 1, 64, 2, True),
]


@pytest.mark.parametrize("m,n,h,arity,two", CASES)
def test_orthonormalize_matches_oracle(cuda_lib, m, n, h, arity, two):
    import paper_0912_2572_gb300 as ts
    A = inputs.gaussian(m, n, seed=61 + n)
    Ad = to_dev(A)
    Q, R = ts.orthonormalize(Ad, leaf_h=h, arity=arity, two_level=two)
    Qh, Rh = to_host(Q), to_host(R)
    Qo, Ro, _ = oracle.qr(A)
    assert np.all(np.diag(Rh) >= 0) and np.all(np.tril(Rh, -1) == 0)
    assert rel(Rh, Ro) <= R_TOL
    assert rel(Qh, Qo) <= R_TOL
    assert oracle.backward_error(A, Qh, Rh) <= BE_TOL
    assert oracle.orth_error(Qh) <= BE_TOL
    assert np.array_equal(to_host(Ad), A)          # out of place: A untouched
    F = ts.factor(Ad, leaf_h=h, arity=arity, two_level=two)
    assert np.array_equal(to_host(F.form_q()), Qh)
    assert np.array_equal(to_host(F.R), Rh)
    F.free()


def test_orthonormalize_in_place(cuda_lib):
    """Q = A: the factorization reads all of A before the thin Q overwrites it."""
    import paper_0912_2572_gb300 as ts
    m, n = 200_003, 32
    A = inputs.graded(m, n, 4.0, seed_g=62, seed_v=63)
    Q1, R1 = ts.orthonormalize(to_dev(A), leaf_h=144, arity=2, two_level=True)
    Ad = to_dev(A)
    Q2, R2 = ts.orthonormalize(Ad, Q=Ad, leaf_h=144, arity=2, two_level=True)
    assert Q2.data_ptr() == Ad.data_ptr()
    assert np.array_equal(to_host(Ad), to_host(Q1))
    assert np.array_equal(to_host(R2), to_host(R1))


def test_block_gram_schmidt_basis(cuda_lib):
    """Block classical Gram-Schmidt with reorthogonalization (BCGS2), TSQR as the
    intra-block step: five blocks of 16 columns of a 100,000-row matrix. Each block is
    projected against the basis and orthonormalized twice. The basis stays orthonormal
    to working precision and spans the blocks (each block is V C for C = V^T X)."""
    import paper_0912_2572_gb300 as ts
    m, b, nb = 100_000, 16, 5
    V = np.zeros((m, 0))
    for q in range(nb):
        X = inputs.gaussian(m, b, seed=700 + q)
        W = X
        for _ in range(2):
            W = W - V @ (V.T @ W)
            Qd, _R = ts.orthonormalize(to_dev(W), leaf_h=256, arity=2)
            W = to_host(Qd)
        V = np.hstack([V, W])
        C = V.T @ X
        assert np.linalg.norm(X - V @ C) / np.linalg.norm(X) <= 1e-13
    assert oracle.orth_error(V) <= 1e-13
