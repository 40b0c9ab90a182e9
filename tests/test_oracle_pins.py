"""Pins of the CPU oracle against facts that do not come from the oracle itself.

The oracle is the plain definition of what TSQR computes: an unblocked FP64
Householder QR (paper §2.2), sign-normalised so that diag(R) >= 0, which makes R and
the thin Q unique for full-rank A (paper §2.2), plus Q^T b, Q b, the thin Q and least
squares. Each test below checks it against something independent:
  * brute force: exact rational arithmetic (R^T R = A^T A by an LDL^T factorization in
    fractions), a Givens-rotation QR and modified Gram-Schmidt in extended precision;
  * closed forms with known R; the combine identity of paper §2.3; invariants;
  * a black-box library routine (LAPACK through numpy) on small inputs;
  * planted mistakes: mutated copies of the oracle source must fail these pins.
"""
import math
import os
import re
import shutil
import subprocess
import sys
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_0912_2572_gb300 import inputs

TOL = 1e-14


def rel(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / (nb if nb > 0 else 1.0)


# ----------------------------------------------------------------- brute force
def exact_r(A):
    """R with diag > 0 from R^T R = A^T A, computed as A^T A = L D L^T in exact
    rationals (integer A); r_jk = sqrt(d_j) L_kj. Only the final square roots and
    products are rounded (about 2 ulp)."""
    m, n = A.shape
    Ai = [[Fraction(int(A[i, j])) for j in range(n)] for i in range(m)]
    G = [[sum(Ai[i][a] * Ai[i][b] for i in range(m)) for b in range(n)] for a in range(n)]
    L = [[Fraction(0)] * n for _ in range(n)]
    d = [Fraction(0)] * n
    for j in range(n):
        d[j] = G[j][j] - sum(L[j][l] ** 2 * d[l] for l in range(j))
        L[j][j] = Fraction(1)
        for i in range(j + 1, n):
            L[i][j] = (G[i][j] - sum(L[i][l] * L[j][l] * d[l] for l in range(j))) / d[j]
    R = np.zeros((n, n))
    for j in range(n):
        s = math.sqrt(float(d[j]))
        for k in range(j, n):
            R[j, k] = s * float(L[k][j])
    return R


def givens_r(A):
    """R by Givens rotations in extended precision (a different algorithm)."""
    X = np.array(A, dtype=np.longdouble)
    m, n = X.shape
    for j in range(n):
        for i in range(m - 1, j, -1):
            a, b = X[i - 1, j], X[i, j]
            if b == 0:
                continue
            r = np.sqrt(a * a + b * b)
            c, s = a / r, b / r
            top = c * X[i - 1, :] + s * X[i, :]
            bot = -s * X[i - 1, :] + c * X[i, :]
            X[i - 1, :], X[i, :] = top, bot
            X[i, j] = 0
    R = np.triu(X[:n, :n])
    sgn = np.where(np.diag(R) < 0, -1, 1).astype(np.longdouble)
    return np.array(R * sgn[:, None], dtype=np.float64)


def mgs(A):
    """Modified Gram-Schmidt in extended precision: (Q, R) with diag(R) > 0."""
    X = np.array(A, dtype=np.longdouble)
    m, n = X.shape
    Q = np.zeros_like(X)
    R = np.zeros((n, n), dtype=np.longdouble)
    for j in range(n):
        v = X[:, j].copy()
        for i in range(j):
            R[i, j] = Q[:, i] @ v
            v = v - R[i, j] * Q[:, i]
        R[j, j] = np.sqrt(v @ v)
        Q[:, j] = v / R[j, j]
    return np.array(Q, dtype=np.float64), np.array(R, dtype=np.float64)


@pytest.mark.parametrize("shape,seed", [((3, 2), 0), ((5, 3), 1), ((8, 4), 2), ((12, 6), 3)])
def test_r_matches_exact_rational(shape, seed):
    A = inputs.integer_matrix(*shape, seed=seed)
    if np.linalg.matrix_rank(A) < shape[1]:
        pytest.skip("rank-deficient draw")
    assert rel(oracle.r_factor(A), exact_r(A)) <= 1e-14


@pytest.mark.parametrize("m,n,seed", [(6, 3, 0), (20, 5, 1), (40, 9, 2)])
def test_r_matches_givens_and_mgs(m, n, seed):
    A = inputs.gaussian(m, n, seed)
    Q, R, _ = oracle.qr(A)
    assert rel(R, givens_r(A)) <= TOL
    Qm, Rm = mgs(A)
    assert rel(R, Rm) <= TOL
    assert rel(Q, Qm) <= TOL


def test_matches_lapack_black_box():
    A = inputs.gaussian(200, 12, 5)
    Q, R, _ = oracle.qr(A)
    q, r = np.linalg.qr(A)
    s = np.where(np.diag(r) < 0, -1.0, 1.0)
    assert rel(R, r * s[:, None]) <= TOL
    assert rel(Q, q * s[None, :]) <= TOL


# ------------------------------------------------------------------ closed forms
def test_closed_form_orthonormal_times_diagonal():
    """A = Q0 diag(d) with orthonormal Q0 has R = diag(|d|) and Q = Q0 sign(d)."""
    Q0 = np.linalg.qr(inputs.gaussian(300, 10, 7))[0]
    d = np.array([3.0, -2.0, 0.5, -7.0, 1.0, 1e-3, -1e3, 2.5, -0.25, 4.0])
    Q, R, _ = oracle.qr(Q0 * d[None, :])
    assert rel(R, np.diag(np.abs(d))) <= TOL
    assert rel(Q, Q0 * np.sign(d)[None, :]) <= TOL


def test_closed_form_upper_triangular():
    """A square upper triangular: R = D A with D = sign(diag A)."""
    U = np.triu(inputs.gaussian(9, 9, 3)) + 5 * np.eye(9) * np.sign(inputs.gaussian(9, 1, 4)[:, 0])[:, None]
    R = oracle.r_factor(U)
    assert rel(R, np.sign(np.diag(U))[:, None] * U) <= TOL


def test_near_triangular_input_is_stable():
    """A nearly upper-triangular matrix (|below-diagonal| ~ 1e-12 |diagonal|) is where a
    reflector with the cancelling sign choice breaks down (alpha - beta ~ 0). The
    backward error must stay at rounding level and R close to D U."""
    U = np.triu(inputs.gaussian(40, 8, 3)[:8]) + 3 * np.eye(8)
    A = np.vstack([U, np.zeros((32, 8))]) + 1e-12 * np.tril(inputs.gaussian(40, 8, 4), -1)
    Q, R, _ = oracle.qr(A)
    assert np.all(np.isfinite(R)) and np.all(np.isfinite(Q))
    assert oracle.backward_error(A, Q, R) <= 1e-14 * 8
    assert oracle.orth_error(Q) <= 1e-14 * 8
    assert rel(R, np.sign(np.diag(U))[:, None] * U) <= 1e-11


def test_closed_form_orthonormal_columns():
    Q0 = np.linalg.qr(inputs.gaussian(100, 8, 9))[0]
    assert rel(oracle.r_factor(Q0), np.eye(8)) <= TOL


def test_closed_form_single_column():
    a = inputs.gaussian(50, 1, 11)
    Q, R, _ = oracle.qr(a)
    nrm = math.sqrt(float(np.sum(a.astype(np.longdouble) ** 2)))
    assert abs(R[0, 0] - nrm) <= 1e-15 * nrm
    assert rel(Q[:, 0], a[:, 0] / nrm) <= TOL


def test_combine_identity_of_stacked_triangles():
    """The TSQR reduce operator (paper §2.3): R([A1; A2]) = R([R(A1); R(A2)])."""
    A1, A2 = inputs.gaussian(60, 7, 1), inputs.gaussian(45, 7, 2)
    R12 = oracle.r_factor(np.vstack([A1, A2]))
    Rc = oracle.r_factor(np.vstack([oracle.r_factor(A1), oracle.r_factor(A2)]))
    assert rel(Rc, R12) <= 1e-14


def test_tree_shape_independence():
    """Associativity (paper §2.3): a binary and a flat reduction of four blocks agree."""
    blocks = [inputs.gaussian(30, 5, s) for s in range(4)]
    Rs = [oracle.r_factor(b) for b in blocks]
    binary = oracle.r_factor(np.vstack([oracle.r_factor(np.vstack(Rs[:2])),
                                        oracle.r_factor(np.vstack(Rs[2:]))]))
    flat = Rs[0]
    for r in Rs[1:]:
        flat = oracle.r_factor(np.vstack([flat, r]))
    assert rel(binary, flat) <= 1e-14
    assert rel(binary, oracle.r_factor(np.vstack(blocks))) <= 1e-14


# -------------------------------------------------------------------- invariants
@pytest.mark.parametrize("m,n,dec", [(500, 16, 0), (400, 32, 6), (1000, 64, 6)])
def test_invariants(m, n, dec):
    A = inputs.graded(m, n, dec) if dec else inputs.gaussian(m, n, 1)
    Q, R, _ = oracle.qr(A)
    assert np.all(np.tril(R, -1) == 0)
    assert np.all(np.diag(R) >= 0)
    assert oracle.backward_error(A, Q, R) <= 1e-14 * n
    assert oracle.orth_error(Q) <= 1e-14 * n
    perm = inputs.rng(3).permutation(m)
    assert rel(oracle.r_factor(A[perm]), R) <= 1e-13


def test_sign_of_zero_and_zero_column():
    """sign(0) = +1, and a zero column gives tau = 0 (H = I) and r_jj = 0."""
    A = inputs.gaussian(10, 3, 1)
    A[:, 1] = 0.0
    Q, R, d = oracle.qr(A)
    assert R[1, 1] == 0.0 and d[1] == 1.0
    assert oracle.backward_error(A, Q, R) <= 1e-15


def test_thin_q_reflector_j_leaves_columns_below_j():
    """Forming the thin Q applies H_{n-1} first: the reflectors j..n-1 leave column c < j of
    [I_n; 0] exactly unchanged, since v_k is zero above row k (§4, Property 1: the thin Q
    costs the factorization's flops, not twice them). Both thin-Q kernels skip those
    columns."""
    m, n = 200, 9
    A = inputs.gaussian(m, n, 6)
    VR, tau = oracle.householder(A)
    E = np.zeros((m, n))
    E[:n, :n] = np.eye(n)
    for j in range(1, n):
        t = tau.copy()
        t[:j] = 0.0                                  # only H_j .. H_{n-1}
        C = oracle.apply_q(VR, t, E)
        assert np.array_equal(C[:, :j], E[:, :j])
        assert not np.array_equal(C[:, j], E[:, j])  # column j is the first one touched


def test_apply_roundtrip_and_thin_part():
    m, n, k = 300, 12, 3
    A = inputs.gaussian(m, n, 4)
    B = inputs.gaussian(m, k, 5)
    VR, tau = oracle.householder(A)
    C = oracle.apply_qt(VR, tau, B)
    assert rel(oracle.apply_q(VR, tau, C), B) <= TOL
    assert abs(np.linalg.norm(C) - np.linalg.norm(B)) <= 1e-14 * np.linalg.norm(B)
    Q, _, _ = oracle.qr(A)
    top, tail = oracle.qt_b(A, B)
    assert rel(top, Q.T @ B) <= TOL
    assert rel(tail, np.linalg.norm(B - Q @ (Q.T @ B), axis=0)) <= 1e-13


# ------------------------------------------------------------------ least squares
def test_lstsq_exact_rational_normal_equations():
    A = inputs.integer_matrix(9, 4, seed=6)
    b = inputs.integer_matrix(9, 1, seed=7)[:, 0]
    Af = [[Fraction(int(v)) for v in row] for row in A]
    bf = [Fraction(int(v)) for v in b]
    n = A.shape[1]
    G = [[sum(Af[i][a] * Af[i][c] for i in range(9)) for c in range(n)] for a in range(n)]
    r = [sum(Af[i][a] * bf[i] for i in range(9)) for a in range(n)]
    M = [G[i][:] + [r[i]] for i in range(n)]  # Gauss-Jordan in rationals
    for c in range(n):
        p = next(i for i in range(c, n) if M[i][c] != 0)
        M[c], M[p] = M[p], M[c]
        M[c] = [v / M[c][c] for v in M[c]]
        for i in range(n):
            if i != c:
                f = M[i][c]
                M[i] = [vi - f * vc for vi, vc in zip(M[i], M[c])]
    x_exact = np.array([float(M[i][n]) for i in range(n)])
    assert rel(oracle.lstsq(A, b), x_exact) <= 1e-13


def test_lstsq_consistent_system_and_lapack():
    A = inputs.graded(800, 10, 3)
    x_true = inputs.gaussian(10, 2, 8)
    assert rel(oracle.lstsq(A, A @ x_true), x_true) <= 1e-11
    b = inputs.gaussian(800, 1, 9)[:, 0]
    assert rel(oracle.lstsq(A, b), np.linalg.lstsq(A, b, rcond=None)[0]) <= 1e-12


def test_mixed_refinement_reaches_fp64_and_x_only_stalls():
    """Bjorck augmented-system refinement around an FP32 QR reaches the FP64 solution
    for kappa ~ 1e4 with a nonzero residual; x-only refinement stalls (negative control)."""
    A = inputs.graded(4000, 16, 4)
    b, _ = inputs.lstsq_rhs(A, 1, 1e-6, 2)
    xo = oracle.lstsq(A, b[:, 0])
    x, r, hist = oracle.lstsq_refine_mixed(A, b[:, 0], max_steps=10)
    assert rel(x, xo) <= 1e-10
    assert hist[-1] <= 1e-13
    assert rel(r, b[:, 0] - A @ x) <= 1e-8
    x2, _ = oracle.lstsq_refine_x_only(A, b[:, 0], max_steps=10)
    assert rel(x2, xo) > 1e-9


# --------------------------------------------------------- error measures, pinned
def exact_orth_error(Q):
    """||Q^T Q - I||_F of a matrix with dyadic entries: the Gram matrix in exact
    rationals (Fraction(float) is exact), one rounding in the final square root."""
    m, n = Q.shape
    Qf = [[Fraction(float(Q[i, j])) for j in range(n)] for i in range(m)]
    s = Fraction(0)
    for a in range(n):
        for b in range(n):
            g = sum(Qf[i][a] * Qf[i][b] for i in range(m)) - (1 if a == b else 0)
            s += g * g
    return math.sqrt(float(s))


def test_orth_error_closed_forms():
    """Q = c [I_n; 0] gives Q^T Q - I = (c^2 - 1) I, an error of sqrt(n) |c^2 - 1|; two
    unit columns at inner product eps give sqrt(2) |eps| (the off-diagonal entry counts
    twice); a Q with orthonormal columns gives 0."""
    for n, c in ((5, 1.5), (8, 0.75), (3, 2.0)):
        Q = np.zeros((20, n))
        Q[:n, :n] = c * np.eye(n)
        expect = math.sqrt(n) * abs(c * c - 1.0)
        assert abs(oracle.orth_error(Q) - expect) <= 1e-15 * expect
    eps = 2.0 ** -12
    Q = np.zeros((4, 2))
    Q[0, 0] = 1.0
    Q[0, 1], Q[1, 1] = eps, math.sqrt(1.0 - eps * eps)
    assert abs(oracle.orth_error(Q) - math.sqrt(2.0) * eps) <= 1e-9 * eps
    E = np.zeros((10, 4))
    E[[2, 5, 7, 9], [0, 1, 2, 3]] = [1.0, -1.0, 1.0, 1.0]
    assert oracle.orth_error(E) == 0.0


def test_orth_error_exact_rational():
    """A dyadic 9-by-4 matrix: every term of ||Q^T Q - I||_F, diagonal and off-diagonal,
    against the exact rational Gram matrix."""
    Q = inputs.integer_matrix(9, 4, seed=12) / 8.0
    assert abs(oracle.orth_error(Q) - exact_orth_error(Q)) <= 1e-14 * exact_orth_error(Q)
    Q2 = np.eye(6, 3) + inputs.integer_matrix(6, 3, seed=13) / 64.0
    assert abs(oracle.orth_error(Q2) - exact_orth_error(Q2)) <= 1e-14 * exact_orth_error(Q2)


def test_trsv_upper_t_exact_rational():
    """R^T x = g (forward substitution) against the exact rational solution for integer R
    with a nonzero diagonal, and x = e_0 / r_00 for g = e_0 (only the first unknown is
    then nonzero when R is diagonal)."""
    n = 7
    R = np.triu(inputs.integer_matrix(n, n, seed=14)).astype(np.float64)
    R[np.arange(n), np.arange(n)] = np.where(np.diag(R) == 0, 3.0, np.diag(R))
    g = inputs.integer_matrix(n, 1, seed=15)[:, 0].astype(np.float64)
    Rf = [[Fraction(int(R[i, j])) for j in range(n)] for i in range(n)]
    x = [Fraction(0)] * n
    for i in range(n):  # column i of R holds row i of R^T
        x[i] = (Fraction(int(g[i])) - sum(Rf[l][i] * x[l] for l in range(i))) / Rf[i][i]
    xe = np.array([float(v) for v in x])
    assert rel(oracle.trsv_upper_t(R, g), xe) <= 1e-14
    D = np.diag(np.arange(1.0, n + 1))
    assert np.array_equal(oracle.trsv_upper_t(D, np.eye(n)[0]), np.eye(n)[0])
    with pytest.raises(np.linalg.LinAlgError):
        Z = R.copy()
        Z[3, 3] = 0.0
        oracle.trsv_upper_t(Z, g)


def test_raw_diagonal_sign_convention():
    """Before sign normalisation, r_00 = -sign(a_00) ||a_0|| in both precisions (the
    reflector's sign choice that avoids cancellation, sign(0) = +1)."""
    A = inputs.gaussian(30, 3, 16)
    for a00 in (2.5, -2.5, 0.0):
        A[0, 0] = a00
        nrm = float(np.linalg.norm(A[:, 0]))
        expect = -(-1.0 if a00 < 0 else 1.0) * nrm
        VR, _ = oracle.householder(A)
        assert abs(VR[0, 0] - expect) <= 1e-15 * nrm
        V32, _ = oracle.geqr2_f32(A)
        assert abs(float(V32[0, 0]) - expect) <= 1e-6 * nrm


# ------------------------------------------------------- the FP32 Householder QR
U32 = 2.0 ** -24


def test_geqr2_f32_against_fp64_and_exact():
    """The FP32 QR of an input exact in FP32 (integers): R within the FP32 backward bound
    of the exact rational R, and not at FP64 accuracy (every operation is FP32)."""
    for shape, seed in (((12, 6), 3), ((40, 8), 17)):
        A = inputs.integer_matrix(*shape, seed=seed).astype(np.float64)
        if np.linalg.matrix_rank(A) < shape[1]:
            continue
        V32, _ = oracle.geqr2_f32(A)
        err = rel(oracle.normalised_r_from(V32), exact_r(A))
        assert 1e-11 < err <= 20 * shape[1] * U32


def test_geqr2_f32_closed_form_and_reflectors():
    """A = Q0 diag(d) (Q0 orthonormal, rounded to FP32) gives |R| = diag(|d|) to FP32
    accuracy; Q^T A from the FP32 reflectors is [R; 0] and Q Q^T b = b, both within the
    FP32 bound."""
    Q0 = np.linalg.qr(inputs.gaussian(200, 8, 18))[0].astype(np.float32).astype(np.float64)
    d = np.array([4.0, -2.0, 1.0, 0.5, -0.25, 3.0, -1.5, 2.0])
    A = (Q0 * d[None, :]).astype(np.float32).astype(np.float64)
    V32, tau = oracle.geqr2_f32(A)
    R = oracle.normalised_r_from(V32)
    assert rel(R, np.diag(np.abs(d))) <= 50 * 8 * U32
    Rraw = np.triu(np.asarray(V32[:8], dtype=np.float64))
    for j in range(8):
        c = oracle.apply_qt_f32(V32, tau, A[:, j])
        assert np.linalg.norm(c[:8] - Rraw[:, j]) <= 50 * U32 * np.linalg.norm(A[:, j])
        assert np.linalg.norm(c[8:]) <= 50 * U32 * np.linalg.norm(A[:, j])
    b = inputs.gaussian(200, 1, 19)[:, 0]
    back = oracle.apply_q_f32(V32, tau, oracle.apply_qt_f32(V32, tau, b))
    assert rel(back, b) <= 50 * U32


def test_geqr2_f32_near_triangular_is_stable():
    """The FP32 analogue of the near-triangular case: below-diagonal entries 1e-5 of the
    diagonal, where the cancelling sign choice loses every digit of alpha - beta."""
    n = 8
    U = np.triu(inputs.gaussian(40, n, 3)[:n]) + 3 * np.eye(n)
    A = np.vstack([U, np.zeros((32, n))]) + 1e-5 * np.tril(inputs.gaussian(40, n, 4), -1)
    A = A.astype(np.float32).astype(np.float64)
    V32, tau = oracle.geqr2_f32(A)
    Rraw = np.triu(np.asarray(V32[:n], dtype=np.float64))
    Q = np.column_stack([oracle.apply_q_f32(V32, tau, np.eye(40)[:, j]) for j in range(n)]).astype(np.float64)
    assert np.all(np.isfinite(Rraw))
    assert rel(Q @ Rraw, A) <= 50 * n * U32
    assert oracle.orth_error(Q) <= 50 * n * U32


# --------------------------------------------------- the mixed-precision TSQR R
def test_r_mixed_single_leaf_and_combine():
    """oracle_r_mixed: with one leaf (h >= m) the FP64 combine of a single triangle leaves it
    unchanged, so R is exactly the FP32 QR's R; with several leaves (a ragged last one) it is
    the FP64 R of the stacked FP32 leaf triangles (paper §2.3's reduce, any tree shape), and
    it lies within the FP32 bound of the FP64 R of A without being FP64-accurate."""
    A = inputs.graded(1000, 12, 2.0, seed_g=21, seed_v=22)
    V32, _ = oracle.geqr2_f32(A)
    assert np.array_equal(oracle.r_mixed(A, h=1000), oracle.normalised_r_from(V32))
    leaves = [A[0:128], A[128:256], A[256:384], A[384:512], A[512:640], A[640:768], A[768:1000]]
    tri = []
    for L in leaves:
        VL, _ = oracle.geqr2_f32(L)
        tri.append(np.triu(np.asarray(VL[:12], dtype=np.float64)))
    Rs = oracle.r_factor(np.vstack(tri))
    Rm = oracle.r_mixed(A, h=128)
    assert rel(Rm, Rs) <= 1e-14
    err = rel(Rm, oracle.r_factor(A))
    assert 1e-11 < err <= 50 * 12 * U32


# ---------------------------------- corrected semi-normal equations (the GPU's refinement)
def test_csne_refinement_reaches_fp64_solution():
    """CSNE iterated around the FP32 R reaches the FP64 least-squares solution for
    kappa ~ 1e4 with a nonzero residual, each correction smaller than the last, within
    a few steps; on a consistent well-conditioned system it returns x_true."""
    A = inputs.graded(4000, 16, 4)
    b, _ = inputs.lstsq_rhs(A, 1, 1e-6, 2)
    xo = oracle.lstsq(A, b[:, 0])
    x, hist = oracle.lstsq_refine_csne(A, b[:, 0], max_steps=10)
    assert rel(x, xo) <= 1e-10
    assert hist[0] == 1.0                     # from x = 0 the first correction is all of x
    assert all(hist[s + 1] < hist[s] for s in range(len(hist) - 1))
    rho = max(hist[s + 1] / hist[s] for s in range(len(hist) - 1))
    assert hist[-1] * rho / (1 - rho) <= 1e-10  # the stop: predicted remaining correction
    x2, hist2 = oracle.lstsq_refine_csne(A, b[:, 0], max_steps=20, tol=1e-30)
    assert rel(x2, xo) <= 1e-12 and hist2[-1] <= 1e-13  # run on to the rounding level
    A2 = inputs.graded(1500, 12, 2)
    x_true = inputs.gaussian(12, 1, 20)[:, 0]
    x2, _ = oracle.lstsq_refine_csne(A2, A2 @ x_true, max_steps=10)
    assert rel(x2, x_true) <= 1e-12


def test_thread_count_does_not_change_results():
    code = ("import numpy as np, oracle; from paper_0912_2572_gb300 import inputs;"
            "Q,R,_=oracle.qr(inputs.gaussian(3000,24,1)); print(repr(float(np.sum(R*np.arange(1,577).reshape(24,24)))))")
    outs = []
    for t in ("1", "4"):
        env = dict(os.environ, OMP_NUM_THREADS=t)
        outs.append(subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True,
                                   cwd=os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                                   check=True).stdout)
    assert outs[0] == outs[1]


# --------------------------------------------------------------- planted mistakes
MUTANTS = {
    "beta_sign": ("double beta = -sgn(alpha) * hypot(alpha, sigma);",
                  "double beta = sgn(alpha) * hypot(alpha, sigma);"),
    "tau_formula": ("tau[j] = (beta - alpha) / beta;", "tau[j] = (beta - alpha) / alpha;"),
    "dropped_pivot_term": ("double w = Bc[j];\n  for (int64_t i = j + 1; i < m; i++) w += AT(V, i, j, ldv) * Bc[i];",
                           "double w = 0.0;\n  for (int64_t i = j + 1; i < m; i++) w += AT(V, i, j, ldv) * Bc[i];"),
    "row_index_off_by_one": ("for (int64_t i = j + 1; i < m; i++) Bc[i] -= AT(V, i, j, ldv) * w;",
                             "for (int64_t i = j + 2; i < m; i++) Bc[i] -= AT(V, i, j, ldv) * w;"),
    "transposed_operand": ("kahan_add(&qr, &cq, AT(Q, i, l, ldq) * AT(R, l, j, ldr));",
                           "kahan_add(&qr, &cq, AT(Q, i, l, ldq) * AT(R, j, l, ldr));"),
    "apply_order": ("for (int64_t j = n - 1; j >= 0; j--) {\n#pragma omp parallel for schedule(static)\n    for (int64_t c = 0; c < k; c++) reflect_column(m, j, V, ldv, tau[j], &AT(B, 0, c, ldb));",
                    "for (int64_t j = 0; j < n; j++) {\n#pragma omp parallel for schedule(static)\n    for (int64_t c = 0; c < k; c++) reflect_column(m, j, V, ldv, tau[j], &AT(B, 0, c, ldb));"),
    "orth_offdiag_weight": ("kahan_add(&s, &c, (a == b ? 1.0 : 2.0) * e * e);",
                            "kahan_add(&s, &c, e * e);"),
    "orth_diagonal_only": ("for (int64_t b = a; b < n; b++) {\n      double g = 0.0, cg = 0.0;",
                           "for (int64_t b = a; b <= a; b++) {\n      double g = 0.0, cg = 0.0;"),
    "orth_identity_dropped": ("double e = (g + cg) - (a == b ? 1.0 : 0.0);", "double e = (g + cg);"),
    "trsv_t_transposed": ("for (int64_t l = 0; l < i; l++) s -= AT(R, l, i, ldr) * x[l];",
                          "for (int64_t l = 0; l < i; l++) s -= AT(R, i, l, ldr) * x[l];"),
    "f32_beta_sign": ("float beta = -(alpha < 0.0f ? -1.0f : 1.0f) * hypotf(alpha, sigma);",
                      "float beta = (alpha < 0.0f ? -1.0f : 1.0f) * hypotf(alpha, sigma);"),
    "f32_tau_formula": ("hypotf(alpha, sigma);\n      tau[j] = (beta - alpha) / beta;",
                        "hypotf(alpha, sigma);\n      tau[j] = (beta - alpha) / alpha;"),
    "f32_dropped_pivot_term": ("float w = Bc[j];", "float w = 0.0f;"),
    "f32_scale_denominator": ("float denom = alpha - beta;", "float denom = beta;"),
    "r_mixed_leaf_remainder": ("const int64_t r0 = l * h, rows = (l == P - 1) ? m - r0 : h;",
                               "const int64_t r0 = l * h, rows = h;"),
    "csne_gradient_sign": ("for (int64_t i = 0; i < m; i++) t += AT(A, i, j, lda) * r[i];\n      y[j] = t;",
                           "for (int64_t i = 0; i < m; i++) t -= AT(A, i, j, lda) * r[i];\n      y[j] = t;"),
    "scale_denominator": ("for (int64_t i = 1; i < m - j; i++) x[i] = x[i] / denom;",
                          "for (int64_t i = 1; i < m - j; i++) x[i] = x[i] / beta;"),
}

PIN_SCRIPT = r"""
import sys, numpy as np
sys.path.insert(0, {root!r})
import oracle
from paper_0912_2572_gb300 import inputs
sys.path.insert(0, {tests!r})
import test_oracle_pins as t
failed = []
def run(name, f):
    try:
        f()
    except BaseException as e:
        failed.append(name)
run("exact", lambda: t.test_r_matches_exact_rational((8, 4), 2))
run("givens", lambda: t.test_r_matches_givens_and_mgs(20, 5, 1))
run("closed", t.test_closed_form_orthonormal_times_diagonal)
run("near_triangular", t.test_near_triangular_input_is_stable)
run("invariants", lambda: t.test_invariants(500, 16, 0))
run("apply", t.test_apply_roundtrip_and_thin_part)
run("lstsq", t.test_lstsq_consistent_system_and_lapack)
run("orth_closed", t.test_orth_error_closed_forms)
run("orth_exact", t.test_orth_error_exact_rational)
run("trsv_t", t.test_trsv_upper_t_exact_rational)
run("raw_sign", t.test_raw_diagonal_sign_convention)
run("f32_exact", t.test_geqr2_f32_against_fp64_and_exact)
run("f32_closed", t.test_geqr2_f32_closed_form_and_reflectors)
run("f32_near_triangular", t.test_geqr2_f32_near_triangular_is_stable)
run("csne", t.test_csne_refinement_reaches_fp64_solution)
run("r_mixed", t.test_r_mixed_single_leaf_and_combine)
print("FAILED:" + ",".join(failed))
"""


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistake_is_caught(name, tmp_path):
    """A mutated copy of the oracle (built in a temporary directory) must fail at
    least one pin: the pins are sensitive to dropped terms, wrong signs or indices
    and transposed operands."""
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    src = open(os.path.join(root, "oracle", "tsqr_oracle.c")).read()
    old, new = MUTANTS[name]
    assert old in src, f"mutation anchor for {name} not found"
    mut_root = tmp_path / "r"
    shutil.copytree(os.path.join(root, "oracle"), mut_root / "oracle",
                    ignore=shutil.ignore_patterns("*.so", "__pycache__"))
    shutil.copytree(os.path.join(root, "paper_0912_2572_gb300"), mut_root / "paper_0912_2572_gb300",
                    ignore=shutil.ignore_patterns("*.so", "__pycache__", "_build", "csrc"))
    (mut_root / "oracle" / "tsqr_oracle.c").write_text(src.replace(old, new, 1))
    script = PIN_SCRIPT.format(root=str(mut_root), tests=os.path.dirname(os.path.abspath(__file__)))
    out = subprocess.run([sys.executable, "-c", script], capture_output=True, text=True,
                         env=dict(os.environ, OMP_NUM_THREADS="2"), timeout=300)
    if out.returncode != 0:
        return  # the mutant crashed: caught
    m = re.search(r"FAILED:(.*)", out.stdout)
    assert m is not None, out.stderr[-2000:]
    assert m.group(1).strip() != "", f"mutant {name} passed every pin"
