"""The FP32 leaf chains of the mixed path (register tiles of 128 rows, one block barrier per
column step), through one-item mixed batches (R only): every width the job's column slots
take (one to eight slots per half-warp, widths that leave some half-warps with no column),
leaf tiles only, ragged last tiles and chains of several tiles. R must be upper triangular
with diag >= 0 and match the FP64 oracle to the FP32 leaves' accuracy: the chains' R is
the exact R of a matrix within a few u_32 ||A|| of A (the tree above them is FP64), so for
these well-conditioned Gaussian matrices the relative difference stays near 1e-6."""
import numpy as np
import pytest

import oracle
from paper_0912_2572_gb300 import inputs
from conftest import to_dev, to_host

pytestmark = pytest.mark.gpu

WIDTHS = [1, 2, 3, 8, 15, 16, 17, 31, 33, 47, 63, 64, 65, 96, 127, 128]


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def mixed_r(A, chain_tiles=0):
    import paper_0912_2572_gb300 as ts
    (R, _), = ts.batch_solve([{"A": to_dev(A), "prec": ts.MIXED}], chain_tiles=chain_tiles)
    return to_host(R)


@pytest.mark.parametrize("n", WIDTHS)
def test_fp32_leaf_widths(cuda_lib, n):
    # rows: one full tile, a ragged single tile, and several chains with a ragged last tile
    for m in sorted({max(n, 128), max(n, 77), 128 * 40 + 77}):
        if m < n:
            continue
        A = inputs.gaussian(m, n, 1000 + n + m)
        R = mixed_r(A)
        assert np.all(np.tril(R, -1) == 0) and np.all(np.diag(R) >= 0)
        err = rel(R, oracle.r_factor(A))
        assert err <= 2e-5, f"m={m} n={n}: {err:.2e}"


@pytest.mark.parametrize("m,n,L", [(128 * 64 + 5, 64, 1), (128 * 64, 128, 2), (200_003, 32, 16)])
def test_fp32_leaf_chain_lengths(cuda_lib, m, n, L):
    """Chains of 4 L tiles (the batch's mixed chains are four times the FP64 length): short
    chains with many FP64 combines, and long ones."""
    A = inputs.graded(m, n, 2.0, seed_g=m % 97, seed_v=n)
    R = mixed_r(A, chain_tiles=L)
    assert rel(R, oracle.r_factor(A)) <= 1e-4


def test_fp32_leaf_zero_column_and_scaled_rows(cuda_lib):
    """A zero column (a reflector with tau = 0 on every tile) and rows scaled over eight
    decades (large and small entries in one tile). With a zero column the R factor is not
    unique below its row, so the check is the one every QR satisfies, R^T R = A^T A, plus
    the rows above the zero column (unique) against the oracle."""
    m, n, z = 128 * 12 + 31, 40, 13
    A = inputs.gaussian(m, n, 77)
    A[:, z] = 0.0
    A *= np.logspace(-4, 4, m)[:, None]
    R = mixed_r(A)
    assert np.all(R[: z + 1, z] == 0.0)
    G = A.T @ A
    assert rel(R.T @ R, G) <= 1e-5
    assert rel(R[:z], oracle.r_factor(A)[:z]) <= 1e-4
