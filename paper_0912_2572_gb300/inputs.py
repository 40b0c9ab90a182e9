"""Seeded synthetic inputs shaped like the paper's tall-skinny workloads.

This module holds no arithmetic of the method: it only draws random matrices, so the
oracle and the CUDA path can read identical bytes. The paper factors synthetic dense
FP64 matrices of up to 33,554,432 rows and 64 to 512 columns (§5.1); no dataset is
involved. Every generator is NumPy's PCG64 with an explicit seed, so the same seed
gives the same bytes on x86 and Arm.

Matrices are returned as Fortran-ordered (column-major) float64 arrays.
"""
from __future__ import annotations

import numpy as np


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def gaussian(m: int, n: int, seed: int) -> np.ndarray:
    """iid N(0, 1) entries, column-major m-by-n."""
    return rng(seed).standard_normal((n, m)).T


def haar_orthogonal(n: int, seed: int) -> np.ndarray:
    """A Haar-distributed n-by-n orthogonal matrix (Mezzadri 2007): the Q factor of a
    seeded Gaussian matrix from LAPACK (numpy.linalg.qr), columns multiplied by the
    signs of R's diagonal."""
    g = rng(seed).standard_normal((n, n))
    q, r = np.linalg.qr(g)
    s = np.where(np.diag(r) < 0, -1.0, 1.0)
    return np.asfortranarray(q * s[None, :])


def log_spectrum(n: int, decades: float) -> np.ndarray:
    """sigma_i = 10^(-decades * i / (n-1)), i = 0..n-1 (sigma_0 = 1)."""
    if n == 1:
        return np.ones(1)
    return 10.0 ** (-decades * np.arange(n) / (n - 1))


def graded(m: int, n: int, decades: float, seed_g: int = 0, seed_v: int = 1,
           chunk_rows: int = 1 << 20) -> np.ndarray:
    """A = G diag(sigma) V^T with G iid N(0,1) (m-by-n), sigma log-spaced from 1 to
    10^-decades, V Haar orthogonal; condition number about 10^decades. Built in row
    chunks so the m-by-n product never needs a second full-size temporary."""
    g = rng(seed_g)
    sigma = log_spectrum(n, decades)
    V = haar_orthogonal(n, seed_v)
    M = (sigma[:, None] * V.T)  # diag(sigma) V^T
    A = np.empty((m, n), order="F")
    for r0 in range(0, m, chunk_rows):
        r1 = min(m, r0 + chunk_rows)
        # row-major draws: the stream does not depend on chunk_rows
        G = g.standard_normal((r1 - r0, n))
        A[r0:r1] = G @ M
    return A


def lstsq_rhs(A: np.ndarray, k: int, noise: float, seed: int):
    """(b, x_true) with x_true iid N(0,1) (n-by-k) and b = A x_true + noise * N(0,1)."""
    g = rng(seed)
    n = A.shape[1]
    x_true = np.asfortranarray(g.standard_normal((k, n)).T)
    b = np.asfortranarray(A @ x_true + noise * g.standard_normal((k, A.shape[0])).T)
    return b, x_true


def integer_matrix(m: int, n: int, seed: int, lo: int = -4, hi: int = 5) -> np.ndarray:
    """Small-integer entries (exact in any precision), for brute-force pins."""
    return np.asfortranarray(rng(seed).integers(lo, hi, size=(m, n)).astype(np.float64))
