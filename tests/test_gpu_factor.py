"""FP64 TSQR factorization on the GPU vs the oracle (paper §2.2-§2.3): R with a
non-negative diagonal, the thin Q, Q^T b, and the backward / orthogonality errors."""
import numpy as np
import pytest

import oracle
from paper_0912_2572_gb300 import inputs
from conftest import to_dev, to_host

pytestmark = pytest.mark.gpu

R_TOL = 1e-12      # relative Frobenius error of R against the oracle
BE_TOL = 1e-13     # ||A - QR||_F / ||A||_F and ||Q^T Q - I||_F


def _rel(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


CASES = [
    # (m, n, leaf_h, arity, two_level)
    (4096, 16, 256, 2, False),
    (4096, 16, 256, 2, True),
    (4096, 16, 256, 4, False),
    (4096, 16, 256, 0, False),
    (3000, 7, 100, 2, False),
    (1000, 33, 64, 3, False),
    (777, 64, 128, 2, False),
    (5000, 64, 208, 2, True),
    (2049, 1, 1, 2, False),
    (130, 128, 128, 2, False),
    (1100, 100, 300, 2, True),
    (64, 64, 64, 2, False),
]


@pytest.mark.parametrize("m,n,h,arity,two", CASES)
def test_factor_matches_oracle(cuda_lib, m, n, h, arity, two):
    import paper_0912_2572_gb300 as ts
    A = inputs.gaussian(m, n, seed=m + n)
    Ad = to_dev(A)
    F = ts.factor(Ad, leaf_h=h, arity=arity, two_level=two)
    Q = F.form_q()
    R = to_host(F.R)
    Qh = to_host(Q)
    Qo, Ro, _ = oracle.qr(A)
    assert np.all(np.diag(R) >= 0)
    assert np.all(np.tril(R, -1) == 0)
    assert _rel(R, Ro) <= R_TOL
    assert _rel(Qh, Qo) <= R_TOL  # well-conditioned: the thin Q is entry-wise unique
    assert oracle.backward_error(A, Qh, R) <= BE_TOL
    assert oracle.orth_error(Qh) <= BE_TOL
    # input untouched (not in place)
    assert np.array_equal(to_host(Ad), A)
    F.free()


def test_fp64_peak_probe_is_plausible(cuda_lib):
    """The roofline denominator: the FP64 FMA throughput of a GB300-class GPU is about
    1.2 TFLOP/s (2 DFMA per clock per SM at about 2 GHz), far below its FP32 rate."""
    import paper_0912_2572_gb300 as ts
    tf = ts.probe_fp64_peak()
    assert 0.3 < tf < 3.0


@pytest.mark.parametrize("n", [1, 8, 16, 17, 24, 32, 48, 64])
def test_three_cta_plan_widths(cuda_lib, n):
    """The default tile of the widths that take three CTAs per SM (tiles of at least 2n
    rows; up to 16 columns the chain launch runs the 64-register build, which lets a fourth
    CTA join where its tile fits), on a ragged m: R and the thin Q against the oracle, and
    the plan is the three-CTA one."""
    import paper_0912_2572_gb300 as ts
    m = 60_013
    info = ts.plan_describe(m, n, 1 << 20)
    assert info["ctas_per_sm"] == 3 and info["tile_rows"] >= 2 * n
    A = inputs.gaussian(m, n, 900 + n)
    F = ts.factor(to_dev(A), leaf_h=info["tile_rows"], arity=2, two_level=True)
    Q = to_host(F.form_q())
    R = to_host(F.R)
    F.free()
    Qo, Ro, _ = oracle.qr(A)
    assert _rel(R, Ro) <= R_TOL
    assert _rel(Q, Qo) <= R_TOL
    assert oracle.orth_error(Q) <= BE_TOL


@pytest.mark.parametrize("scale", [1e100, 1e-100, 1e140, 1e-140])
def test_factor_near_the_edges_of_the_supported_range(cuda_lib, scale):
    """Entries are squared without rescaling, so the supported range is about 1e-150..1e150
    (the header's numerical range): matrices scaled by 1e+-100 and 1e+-140 factor to the
    oracle's R (which scales its norms) and an orthonormal Q, the least-squares solution is
    the unscaled one divided by the scale."""
    import paper_0912_2572_gb300 as ts
    m, n = 20_000, 24
    A0 = inputs.graded(m, n, 3.0, seed_g=77, seed_v=78)
    A = A0 * scale
    Ad = to_dev(A)
    F = ts.factor(Ad, leaf_h=144)
    R, Q = to_host(F.R), to_host(F.form_q())
    F.free()
    Ro = oracle.r_factor(A)
    assert np.all(np.isfinite(R)) and np.all(np.isfinite(Q))
    assert _rel(R, Ro) <= R_TOL
    assert oracle.orth_error(Q) <= BE_TOL
    b = inputs.gaussian(m, 1, 79)
    x = to_host(ts.lstsq(Ad, to_dev(b), leaf_h=144))
    xo = oracle.lstsq(A0, b)
    assert _rel(x * scale, xo) <= 1e-11
