"""The host-buffer entry point tsqr_qr_solve_host: the whole FP64 path (copies in, TSQR
factorization, thin Q, Q^T B and the solve, copies out) in one stream-ordered call. Its
results must be bitwise those of the device-pointer calls (tsqr_factor, tsqr_form_q,
tsqr_apply_qt, tsqr_solve_r: the same kernels on the same data) and match the oracle,
with pinned and with pageable host memory."""
import numpy as np
import pytest

import oracle
from paper_0912_2572_gb300 import inputs
from conftest import to_dev, to_host

pytestmark = pytest.mark.gpu


def host(a, pinned):
    import torch
    t = torch.empty((a.shape[1], a.shape[0]), dtype=torch.float64, pin_memory=pinned)
    t.numpy()[:] = a.T
    return t.t()


@pytest.mark.parametrize("m,n,k,pinned", [(50_000, 32, 2, True), (30_000, 64, 1, False), (777, 9, 3, True)])
def test_host_buffers_match_device_path_and_oracle(cuda_lib, m, n, k, pinned):
    import torch
    import paper_0912_2572_gb300 as ts
    A = inputs.graded(m, n, 3.0, seed_g=m % 97, seed_v=5)
    B, _ = inputs.lstsq_rhs(A, k, 1e-4, 6)
    Ah, Bh = host(A, pinned), host(B, pinned)
    Qh = host(np.zeros((m, n)), pinned)
    Rh = host(np.zeros((n, n)), pinned)
    Xh = host(np.zeros((n, k)), pinned)
    st = torch.zeros(1, dtype=torch.int32).pin_memory()
    ts.qr_solve_host(Ah, Bh, Q=Qh, R=Rh, X=Xh, leaf_h=256, status=st)
    torch.cuda.synchronize()
    assert int(st[0]) == 0
    Ad = to_dev(A)
    F = ts.factor(Ad, leaf_h=256)
    Q = to_host(F.form_q())
    C = to_dev(B)
    F.apply_qt(C)
    X = to_host(F.solve_r(C))
    R = to_host(F.R)
    F.free()
    assert np.array_equal(Qh.numpy(), Q) and np.array_equal(Rh.numpy(), R) and np.array_equal(Xh.numpy(), X)
    Qo, Ro, _ = oracle.qr(A)
    assert np.linalg.norm(R - Ro) / np.linalg.norm(Ro) <= 1e-12
    assert np.linalg.norm(Xh.numpy() - oracle.lstsq(A, B)) / np.linalg.norm(oracle.lstsq(A, B)) <= 1e-10
    assert oracle.orth_error(Qh.numpy()) <= 1e-13


def test_host_buffers_optional_outputs_events_and_singular(cuda_lib):
    """R only (no B, no Q); the after/done events order two calls' kernels; a zero column
    reports a singular R through the status word."""
    import torch
    import paper_0912_2572_gb300 as ts
    m, n = 10_000, 16
    A = inputs.gaussian(m, n, 7)
    Rh = host(np.zeros((n, n)), True)
    done = torch.cuda.Event()
    done.record()
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    ts.qr_solve_host(host(A, True), R=Rh, leaf_h=128, stream=s1, done=done)
    Rh2 = host(np.zeros((n, n)), True)
    ts.qr_solve_host(host(A, True), R=Rh2, leaf_h=128, stream=s2, after=done)
    torch.cuda.synchronize()
    assert np.array_equal(Rh.numpy(), Rh2.numpy())
    assert np.linalg.norm(Rh.numpy() - oracle.r_factor(A)) / np.linalg.norm(Rh.numpy()) <= 1e-12
    A[:, 4] = 0.0
    B = inputs.gaussian(m, 1, 8)
    st = torch.zeros(1, dtype=torch.int32).pin_memory()
    Xh = host(np.zeros((n, 1)), True)
    ts.qr_solve_host(host(A, True), host(B, True), X=Xh, leaf_h=128, status=st)
    torch.cuda.synchronize()
    assert int(st[0]) == 4
