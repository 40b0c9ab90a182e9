"""CAQR on the GPU vs the oracle (paper §2.4; the switch from TSQR to CAQR for wide
matrices in §6 and Property 5 of §4): panels of TSQR, each panel's Q^T applied to the
trailing columns. The oracle is the same plain Householder QR of the whole matrix, so R
(diag >= 0), the thin Q, Q^T b and x are compared with it directly, plus the backward and
orthogonality errors."""
import numpy as np
import pytest

import oracle
from paper_0912_2572_gb300 import inputs
from conftest import to_dev, to_host

pytestmark = pytest.mark.gpu

R_TOL = 1e-12      # relative Frobenius error of R (and of the thin Q, well conditioned)
BE_TOL = 1e-13     # ||A - QR||_F / ||A||_F and ||Q^T Q - I||_F


def _rel(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


CASES = [
    # (m, n, panel, leaf_h, arity, two_level): several panels, a ragged last panel, a
    # square matrix, 128-column panels, a flat tree per panel
    (6000, 256, 64, 256, 2, True),
    (4000, 512, 128, 256, 2, True),
    (3000, 200, 48, 96, 4, False),
    (300, 300, 64, 64, 2, False),
    (2500, 130, 0, 256, 0, False),
]


@pytest.mark.parametrize("m,n,panel,h,arity,two", CASES)
def test_caqr_matches_oracle(cuda_lib, m, n, panel, h, arity, two):
    import paper_0912_2572_gb300 as ts
    A = inputs.gaussian(m, n, seed=m + n + panel)
    Ad = to_dev(A)
    F = ts.caqr(Ad, panel=panel, leaf_h=h, arity=arity, two_level=two)
    Q = F.form_q()
    R, Qh = to_host(F.R), to_host(Q)
    Qo, Ro, _ = oracle.qr(A)
    assert np.all(np.diag(R) >= 0)
    assert np.all(np.tril(R, -1) == 0)
    assert _rel(R, Ro) <= R_TOL
    if m > n:  # the square case's last columns of Q are as ill-determined as its last rows of R
        assert _rel(Qh, Qo) <= R_TOL
    assert oracle.backward_error(A, Qh, R) <= BE_TOL
    assert oracle.orth_error(Qh) <= BE_TOL
    assert np.array_equal(to_host(Ad), A)  # not in place: A untouched
    info = F.info()
    assert info["m"] == m and info["n"] == n
    F.free()


def test_caqr_graded_matrix(cuda_lib):
    """kappa = 1e6 (the headline matrix's spectrum) at 20,000 x 256: R against the oracle
    and the kappa-free backward and orthogonality errors."""
    import paper_0912_2572_gb300 as ts
    m, n = 20000, 256
    A = inputs.graded(m, n, 6.0, seed_g=40, seed_v=41)
    F = ts.caqr(to_dev(A), panel=64, leaf_h=256)
    Qh, R = to_host(F.form_q()), to_host(F.R)
    Ro = oracle.r_factor(A)
    assert _rel(R, Ro) <= R_TOL
    assert oracle.backward_error(A, Qh, R) <= BE_TOL
    assert oracle.orth_error(Qh) <= BE_TOL
    F.free()


def test_caqr_apply_and_least_squares(cuda_lib):
    """Q^T B's unique part (top n rows and the norms of the rest) and Q Q^T B = B, then
    tsqr_lstsq with n > 128 (CAQR inside) and solve_r after apply_qt, against the oracle."""
    import torch
    import paper_0912_2572_gb300 as ts
    m, n, k = 5000, 192, 3
    A = inputs.graded(m, n, 2.0, seed_g=42, seed_v=43)
    B, _ = inputs.lstsq_rhs(A, k, 1e-3, 44)
    F = ts.caqr(to_dev(A), panel=64, leaf_h=256)
    C = to_dev(B)
    F.apply_qt(C)
    top, tail = oracle.qt_b(A, B)
    Ch = to_host(C)
    assert _rel(Ch[:n], top) <= R_TOL
    assert _rel(np.linalg.norm(Ch[n:], axis=0), tail) <= R_TOL
    F.apply_q(C)
    assert _rel(to_host(C), B) <= 1e-14 * n
    C2 = to_dev(B)
    F.apply_qt(C2)
    X1 = to_host(F.solve_r(C2))
    Xo = oracle.lstsq(A, B)
    assert _rel(X1, Xo) <= R_TOL
    X2 = to_host(ts.lstsq(to_dev(A), to_dev(B), leaf_h=256))
    assert _rel(X2, Xo) <= R_TOL
    F.free()
    with pytest.raises(ts.TSQRError):  # the mixed path takes n <= 128
        ts.lstsq(to_dev(A), to_dev(B), leaf_h=256, prec=ts.MIXED)
    torch.cuda.synchronize()


def test_caqr_in_place_and_orthonormalize_bitwise(cuda_lib):
    """The in-place factorization and tsqr_orthonormalize with n > 128 run the same
    launches on the same data: R and the thin Q are bitwise those of the out-of-place
    tsqr_caqr + tsqr_form_q."""
    import paper_0912_2572_gb300 as ts
    m, n = 3000, 160
    A = inputs.gaussian(m, n, 45)
    F = ts.caqr(to_dev(A), leaf_h=256)
    Q, R = to_host(F.form_q()), to_host(F.R)
    F.free()
    Ai = to_dev(A)
    Fi = ts.caqr(Ai, leaf_h=256, inplace=True)
    assert np.array_equal(to_host(Fi.R), R)
    assert np.array_equal(to_host(Fi.form_q()), Q)
    Fi.free()
    Q2, R2 = ts.orthonormalize(to_dev(A), leaf_h=256)
    assert np.array_equal(to_host(Q2), Q)
    assert np.array_equal(to_host(R2), R)
    Ab = to_dev(A)
    ts.orthonormalize(Ab, Q=Ab, leaf_h=256)  # in place over A
    assert np.array_equal(to_host(Ab), Q)


def test_caqr_panel_width_does_not_change_the_answer(cuda_lib):
    """Panels of 32, 64 and 128 columns give the same R to rounding (R is unique)."""
    import paper_0912_2572_gb300 as ts
    m, n = 4000, 256
    A = inputs.gaussian(m, n, 46)
    Rs = []
    for panel in (32, 64, 128):
        F = ts.caqr(to_dev(A), panel=panel, leaf_h=256)
        Rs.append(to_host(F.R))
        F.free()
    assert _rel(Rs[0], Rs[2]) <= R_TOL and _rel(Rs[1], Rs[2]) <= R_TOL
