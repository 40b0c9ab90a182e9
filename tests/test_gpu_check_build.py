"""The bounds-checked build (libtsqr_check.so, compiled with -DTSQR_CHECK): every kernel
checks each job and tile descriptor against its buffers' bounds before using it and, on a
failure, sets a bit of the device error word instead of trapping. Small shapes of every
kernel (factor chains and tree levels, the cluster tier, the warp and tile apply kernels,
the thin Q, CAQR panels, the batched engine with refinement, the static-scratch solve) run
through that build's C ABI; the error word must stay clear and the results must be bitwise
those of the normal build (the checks read descriptors only)."""
import ctypes

import numpy as np
import pytest

from paper_0912_2572_gb300 import inputs
from conftest import to_dev, to_host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def checked():
    from paper_0912_2572_gb300 import build, _lib
    build.build(check=True)
    return _lib.load_checked()


def run_path(lib, A, B, m, n, k, leaf_h, arity, flags, wide=False):
    """factor (or CAQR), thin Q, Q^T B, solve through `lib`; returns host arrays."""
    import torch
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    Ad, Bd = to_dev(A), to_dev(B)
    R = torch.zeros((n, n), dtype=torch.float64, device="cuda").t()
    Q = torch.zeros((n, m), dtype=torch.float64, device="cuda").t()
    X = torch.zeros((k, n), dtype=torch.float64, device="cuda").t()
    h = ctypes.c_void_p()
    if wide:
        st = lib.tsqr_caqr(Ad.data_ptr(), m, n, m, 64, leaf_h, arity, flags, s, ctypes.byref(h), R.data_ptr(), n)
    else:
        st = lib.tsqr_factor(Ad.data_ptr(), m, n, m, leaf_h, arity, 0, flags, s, ctypes.byref(h), R.data_ptr(), n)
    assert st == 0, lib.tsqr_last_error()
    assert lib.tsqr_form_q(h, Q.data_ptr(), m, s) == 0
    assert lib.tsqr_apply_qt(h, Bd.data_ptr(), m, k, s) == 0
    assert lib.tsqr_solve_r(h, Bd.data_ptr(), m, k, X.data_ptr(), n, None, s) == 0
    assert lib.tsqr_free(h) == 0
    torch.cuda.synchronize()
    return to_host(R), to_host(Q), to_host(X)


CASES = [
    # (m, n, k, leaf_h, arity, flags, wide): two-level, pure binary with a ragged tail,
    # 4-ary, flat, the cluster tier, the warp apply (k <= 8) and the tile apply (k > 8),
    # thin Q by passes (n <= 32) and by tiles, CAQR, the tile-pair apply (k = 1)
    (20_000, 32, 3, 144, 2, 2, False),
    (5_003, 16, 12, 100, 2, 0, False),
    (9_000, 64, 1, 256, 4, 0, False),
    (2_000, 8, 2, 64, 0, 0, False),
    (60_000, 48, 2, 64, 2, 4, False),
    (3_000, 200, 2, 144, 2, 2, True),
    (2_000, 8, 1, 64, 0, 0, False),  # one column over a flat tree: the tile-pair apply
]


@pytest.mark.parametrize("m,n,k,h,arity,flags,wide", CASES)
def test_checked_build_is_clean_and_bitwise(cuda_lib, checked, m, n, k, h, arity, flags, wide):
    A = inputs.gaussian(m, n, m + n)
    B = inputs.gaussian(m, k, m + n + 1)
    w = ctypes.c_int32(0)
    assert checked.tsqr_error_word(None, ctypes.byref(w)) in (0, 5)  # clear
    got = run_path(checked, A, B, m, n, k, h, arity, flags, wide)
    assert checked.tsqr_error_word(None, ctypes.byref(w)) == 0 and w.value == 0
    ref = run_path(cuda_lib, A, B, m, n, k, h, arity, flags, wide)
    for a, b in zip(got, ref):
        assert np.array_equal(a, b)


def test_checked_build_batched_and_static(cuda_lib, checked):
    """The persistent batched kernel (FP64 and mixed items, refinement launches) and the
    static-scratch solve under the checked build."""
    import torch
    from paper_0912_2572_gb300 import _lib
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    keep = []
    arr = (_lib.BatchItem * 6)()
    for q in range(6):
        m, n, k = 3000 + 1700 * q, (8, 16, 32, 64, 100, 128)[q], (1, 2, 3, 0, 4, 2)[q]
        A = to_dev(inputs.graded(m, n, 2.0, seed_g=q, seed_v=q + 50))
        B = to_dev(inputs.gaussian(m, max(k, 1), q + 100))
        R = torch.zeros((n, n), dtype=torch.float64, device="cuda").t()
        X = torch.zeros((max(k, 1), n), dtype=torch.float64, device="cuda").t()
        keep += [A, B, R, X]
        arr[q].A, arr[q].m, arr[q].n, arr[q].lda = A.data_ptr(), m, n, m
        arr[q].B, arr[q].ldb, arr[q].k = (B.data_ptr() if k else None), m, k
        arr[q].R, arr[q].ldr = R.data_ptr(), n
        arr[q].X, arr[q].ldx = (X.data_ptr() if k else None), n
        arr[q].prec = q % 2 if n + k <= 144 else 1
    st = (ctypes.c_int32 * 6)()
    assert checked.tsqr_batch_solve(arr, 6, 8, 2, s, st, None) == 0, checked.tsqr_last_error()
    assert list(st) == [0] * 6
    A = to_dev(inputs.gaussian(20_000, 24, 7))
    B = to_dev(inputs.gaussian(20_000, 2, 8))
    X = torch.zeros((2, 24), dtype=torch.float64, device="cuda").t()
    assert checked.tsqr_lstsq_static(A.data_ptr(), 20_000, 24, 20_000, B.data_ptr(), 20_000, 2, X.data_ptr(), 24,
                                     s) == 0
    w = ctypes.c_int32(0)
    assert checked.tsqr_error_word(s, ctypes.byref(w)) == 0 and w.value == 0
