"""GB300 (sm_103a) tall-skinny QR — Python binding of the C-ABI library libtsqr.so.

TSQR (paper §2.3): the rows of a tall m-by-n matrix are split into leaves (domains),
each leaf is factored by Householder reflections (paper §2.2), and the leaves' R factors
are reduced by a tree whose operator is "QR of stacked triangles, keep R". The same
names as the C ABI (include/tsqr.h): factor, apply_qt, apply_q, form_q, lstsq.

This module only marshals arguments: PyTorch provides device memory and the current
stream; every step of the computation runs in the library's CUDA kernels. Matrices are
column-major float64 CUDA tensors of shape (rows, cols) with stride(0) == 1; use
``colmajor`` to obtain one.
"""
from __future__ import annotations

import ctypes

from . import _lib

__all__ = ["FP64", "MIXED", "INPLACE", "TWO_LEVEL", "Factors", "factor", "caqr", "lstsq", "colmajor",
           "TSQRError", "profile_collect", "plan_describe", "batch_solve", "batch_autotune", "factor_autotune",
           "AUTO", "BatchPlan", "Server", "probe_fp64_peak", "orthonormalize", "CLUSTER", "error_word",
           "qr_solve_host", "set_mixed_wy_min_n", "probe_dmma_peak"]

FP64 = 0
MIXED = 1
AUTO = 2
INPLACE = 1
TWO_LEVEL = 2
CLUSTER = 4
TSQRError = _lib.TSQRError


def colmajor(t):
    """A column-major (Fortran-ordered) copy of a 2-D tensor, or t itself if it already is."""
    if t.dim() == 2 and t.stride(0) == 1 and t.stride(1) >= max(1, t.shape[0]):
        return t
    return t.t().contiguous().t()


def _stream(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _check_mat(t, name, rows=None, cols=None):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.float64 or t.dim() != 2:
        raise TypeError(f"{name} must be a 2-D float64 CUDA tensor")
    if t.stride(0) != 1:
        raise ValueError(f"{name} must be column-major (stride(0) == 1); use colmajor()")
    if rows is not None and t.shape[0] != rows:
        raise ValueError(f"{name} has {t.shape[0]} rows, expected {rows}")
    if cols is not None and t.shape[1] != cols:
        raise ValueError(f"{name} has {t.shape[1]} columns, expected {cols}")
    return max(t.stride(1), max(1, t.shape[0]))


class Factors:
    """A factor set: the implicit Q (reflectors of every leaf and tree node) and R."""

    def __init__(self, handle, m, n, R, A_ref, stream):
        self._h = handle
        self.m, self.n = m, n
        self.R = R
        self._A_ref = A_ref  # keeps in-place reflector storage alive
        self._stream = stream

    @property
    def handle(self):
        return self._h

    def info(self) -> dict:
        out = (ctypes.c_int64 * 8)()
        _lib.check(_lib.load().tsqr_factors_info(self._h, out), "tsqr_factors_info")
        keys = ["m", "n", "leaves", "tile_rows", "jobs", "tiles", "launches", "ctas_per_sm"]
        return dict(zip(keys, list(out)))

    def apply_qt(self, B, stream=None):
        """B <- Q^T B in place (B: m-by-k column-major)."""
        ldb = _check_mat(B, "B", rows=self.m)
        _lib.check(_lib.load().tsqr_apply_qt(self._h, B.data_ptr(), ldb, B.shape[1], _stream(stream)),
                   "tsqr_apply_qt")
        return B

    def apply_q(self, B, stream=None):
        """B <- Q B in place."""
        ldb = _check_mat(B, "B", rows=self.m)
        _lib.check(_lib.load().tsqr_apply_q(self._h, B.data_ptr(), ldb, B.shape[1], _stream(stream)),
                   "tsqr_apply_q")
        return B

    def form_q(self, Q=None, stream=None):
        """The thin Q (m-by-n, orthonormal columns, A = Q R with diag(R) >= 0)."""
        import torch
        if Q is None:
            Q = torch.empty((self.n, self.m), dtype=torch.float64, device="cuda").t()
        ldq = _check_mat(Q, "Q", rows=self.m, cols=self.n)
        _lib.check(_lib.load().tsqr_form_q(self._h, Q.data_ptr(), ldq, _stream(stream)), "tsqr_form_q")
        return Q

    def solve_r(self, C, X=None, status=None, stream=None):
        """X = R^{-1} C[0:n] (C as returned by apply_qt); status: optional int32 CUDA
        tensor set to 4 when R has a zero diagonal entry."""
        import torch
        ldc = _check_mat(C, "C")
        k = C.shape[1]
        if X is None:
            X = torch.empty((k, self.n), dtype=torch.float64, device="cuda").t()
        ldx = _check_mat(X, "X", rows=self.n, cols=k)
        sp = status.data_ptr() if status is not None else None
        _lib.check(_lib.load().tsqr_solve_r(self._h, C.data_ptr(), ldc, k, X.data_ptr(), ldx, sp,
                                            _stream(stream)), "tsqr_solve_r")
        return X

    def free(self):
        if self._h:
            _lib.load().tsqr_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def factor(A, leaf_h: int = 256, arity: int = 2, two_level: bool = True, inplace: bool = False,
           R=None, stream=None, qt=None, cluster: bool = False) -> Factors:
    """TSQR factorization of a column-major m-by-n float64 CUDA tensor A (paper §2.3).

    leaf_h: rows per leaf; arity: 2..16 (k-ary tree) or 0 (flat); two_level: a flat chain
    inside each CTA followed by the arity-k tree across CTAs. Returns a Factors object
    whose ``R`` (n-by-n, diag >= 0) is valid once the stream reaches this point. With
    ``qt`` (an m-by-k column-major tensor), also qt <- Q^T qt, overlapped with the
    factorization's tree (tsqr_factor_qt; not with ``inplace``). ``cluster`` (binary
    trees) runs the tree's levels three at a time in thread-block clusters, pipelined
    through distributed shared memory (TSQR_CLUSTER).
    """
    import torch
    lib = _lib.load()
    lda = _check_mat(A, "A")
    m, n = A.shape
    if R is None:
        R = torch.empty((n, n), dtype=torch.float64, device=A.device).t()
    ldr = _check_mat(R, "R", rows=n, cols=n)
    flags = (INPLACE if inplace else 0) | (TWO_LEVEL if two_level else 0) | (CLUSTER if cluster else 0)
    h = ctypes.c_void_p()
    if qt is None:
        st = lib.tsqr_factor(A.data_ptr(), m, n, lda, leaf_h, arity, FP64, flags, _stream(stream),
                             ctypes.byref(h), R.data_ptr(), ldr)
        _lib.check(st, "tsqr_factor")
    else:
        ldq = _check_mat(qt, "qt", rows=m)
        st = lib.tsqr_factor_qt(A.data_ptr(), m, n, lda, qt.data_ptr(), ldq, qt.shape[1], leaf_h, arity, FP64,
                                flags, _stream(stream), ctypes.byref(h), R.data_ptr(), ldr)
        _lib.check(st, "tsqr_factor_qt")
    return Factors(h, m, n, R, A if inplace else None, stream)


def caqr(A, panel: int = 0, leaf_h: int = 256, arity: int = 2, two_level: bool = True, inplace: bool = False,
         R=None, stream=None, cluster: bool = False) -> Factors:
    """CAQR factorization (tsqr_caqr, paper §2.4) of a column-major m-by-n float64 CUDA
    tensor A with n up to 4096: TSQR of panels of ``panel`` columns (0 = 64), each panel's
    Q^T applied to the trailing columns. Returns a Factors object (apply_qt, apply_q,
    form_q, solve_r work as for ``factor``) whose ``R`` is n-by-n with diag >= 0."""
    import torch
    lib = _lib.load()
    lda = _check_mat(A, "A")
    m, n = A.shape
    if R is None:
        R = torch.empty((n, n), dtype=torch.float64, device=A.device).t()
    ldr = _check_mat(R, "R", rows=n, cols=n)
    flags = (INPLACE if inplace else 0) | (TWO_LEVEL if two_level else 0) | (CLUSTER if cluster else 0)
    h = ctypes.c_void_p()
    _lib.check(lib.tsqr_caqr(A.data_ptr(), m, n, lda, panel, leaf_h, arity, flags, _stream(stream), ctypes.byref(h),
                             R.data_ptr(), ldr), "tsqr_caqr")
    return Factors(h, m, n, R, A if inplace else None, stream)


def orthonormalize(A, Q=None, R=None, leaf_h: int = 256, arity: int = 2, two_level: bool = True,
                   stream=None, cluster: bool = False):
    """Q-only TSQR (tsqr_orthonormalize): an orthonormal basis of the columns of the
    column-major m-by-n float64 CUDA tensor A, A = Q R with diag(R) >= 0, the
    orthogonalization step of block iterative methods (paper §2.5, §6). ``Q=A``
    orthonormalizes A in place. Returns (Q, R)."""
    import torch
    lib = _lib.load()
    lda = _check_mat(A, "A")
    m, n = A.shape
    if Q is None:
        Q = torch.empty((n, m), dtype=torch.float64, device=A.device).t()
    ldq = _check_mat(Q, "Q", rows=m, cols=n)
    if R is None:
        R = torch.empty((n, n), dtype=torch.float64, device=A.device).t()
    ldr = _check_mat(R, "R", rows=n, cols=n)
    flags = (TWO_LEVEL if two_level else 0) | (CLUSTER if cluster else 0)
    _lib.check(lib.tsqr_orthonormalize(A.data_ptr(), m, n, lda, Q.data_ptr(), ldq, R.data_ptr(), ldr, leaf_h,
                                       arity, FP64, flags, _stream(stream)), "tsqr_orthonormalize")
    return Q, R


PROFILE_KINDS = {0: "factor_chains", 1: "factor_tree", 2: "apply_qt", 3: "apply_q", 4: "form_q",
                 5: "small", 6: "batch", 7: "refine"}


def _fill_item(slot, it):
    """Fills one tsqr_batch_item from a request dict; returns (tensors to keep alive,
    (R, X) outputs)."""
    import torch
    A = it["A"]
    lda = _check_mat(A, "A")
    m, n = A.shape
    B = it.get("B")
    k = 0
    ldb = m
    X = it.get("X")
    if B is not None:
        ldb = _check_mat(B, "B", rows=m)
        k = B.shape[1]
        if X is None:
            X = torch.empty((k, n), dtype=torch.float64, device=A.device).t()
    R = it.get("R")
    if R is None and it.get("want_r", True):
        R = torch.empty((n, n), dtype=torch.float64, device=A.device).t()
    slot.A = A.data_ptr()
    slot.m, slot.n, slot.lda = m, n, lda
    slot.B = B.data_ptr() if B is not None else None
    slot.ldb, slot.k = ldb, k
    slot.R = R.data_ptr() if R is not None else None
    slot.ldr = _check_mat(R, "R", rows=n, cols=n) if R is not None else n
    slot.X = X.data_ptr() if X is not None else None
    slot.ldx = _check_mat(X, "X", rows=n, cols=k) if X is not None else n
    slot.prec = it.get("prec", FP64)
    return [A, B, R, X], (R, X if k else None)


def batch_solve(items, chain_tiles: int = 0, arity: int = 0, stream=None, status: bool = False,
                info: bool = False):
    """Factor (and solve) many independent problems in one persistent launch.

    items: list of dicts with "A" (m-by-n column-major float64 CUDA tensor) and optional
    "B" (m-by-k), "R" and "X" output tensors (allocated here when missing and "want_r" /
    B are given) and "prec" (FP64, MIXED or AUTO). Returns the list of
    (R, X) per item (None where not requested); with ``status`` also the per-item status
    codes, and with ``info`` the per-item (refinement steps, last ||dX||/||X||) (both
    synchronize the stream).
    """
    lib = _lib.load()
    arr = (_lib.BatchItem * max(1, len(items)))()
    keep = []
    outs = []
    for q, it in enumerate(items):
        kp, out = _fill_item(arr[q], it)
        keep += kp
        outs.append(out)
    st = (ctypes.c_int32 * max(1, len(items)))() if status else None
    inf = (ctypes.c_double * max(2, 2 * len(items)))() if info else None
    _lib.check(lib.tsqr_batch_solve(arr, len(items), chain_tiles, arity, _stream(stream), st, inf),
               "tsqr_batch_solve")
    ret = [outs]
    if status:
        ret.append([st[q] for q in range(len(items))])
    if info:
        ret.append([(int(inf[2 * q]), inf[2 * q + 1]) for q in range(len(items))])
    return ret[0] if len(ret) == 1 else tuple(ret)


# candidate order of tsqr_batch_autotune's time table: chain tiles outer, arity inner
BATCH_TUNE_CANDIDATES = [(L, a) for L in (2, 4, 8, 16, 32) for a in (2, 4)]


def batch_autotune(items, sample: int = 0, stream=None):
    """Picks the batched engine's chain length and tree arity by timing every candidate
    on the first ``sample`` items (0 = up to 1000) with the library's native autotuner
    (tsqr_batch_autotune; synchronizes the stream). Returns (chain_tiles, arity,
    {(chain_tiles, arity): ms})."""
    lib = _lib.load()
    arr = (_lib.BatchItem * max(1, len(items)))()
    keep = []
    for q, it in enumerate(items):
        kp, _ = _fill_item(arr[q], it)
        keep += kp
    L = ctypes.c_int32(0)
    ar = ctypes.c_int32(0)
    table = (ctypes.c_float * len(BATCH_TUNE_CANDIDATES))()
    _lib.check(lib.tsqr_batch_autotune(arr, len(items), sample, _stream(stream), ctypes.byref(L),
                                       ctypes.byref(ar), table), "tsqr_batch_autotune")
    return L.value, ar.value, {c: table[q] for q, c in enumerate(BATCH_TUNE_CANDIDATES)}


def factor_autotune(A, stream=None) -> dict:
    """Picks leaf height, tree arity and tree form for tsqr_factor of A by timing the
    candidates on A itself (tsqr_factor_autotune; A is not modified, the stream is
    synchronized). Returns {"leaf_h", "arity", "two_level", "ms"}."""
    lib = _lib.load()
    lda = _check_mat(A, "A")
    m, n = A.shape
    h = ctypes.c_int32(0)
    ar = ctypes.c_int32(0)
    fl = ctypes.c_int32(0)
    ms = ctypes.c_float(0.0)
    _lib.check(lib.tsqr_factor_autotune(A.data_ptr(), m, n, lda, _stream(stream), ctypes.byref(h),
                                        ctypes.byref(ar), ctypes.byref(fl), ctypes.byref(ms)),
               "tsqr_factor_autotune")
    return {"leaf_h": h.value, "arity": ar.value, "two_level": bool(fl.value & TWO_LEVEL), "ms": ms.value}


class BatchPlan:
    """A batch planned once and replayed as a CUDA graph (tsqr_batch_plan_*).

    items: as for batch_solve. The plan keeps the tensors alive; overwrite the A and B
    tensors in place between runs to solve new data. ``outputs`` is the list of (R, X).
    """

    def __init__(self, items, chain_tiles: int = 0, arity: int = 0):
        self._lib = _lib.load()
        arr = (_lib.BatchItem * max(1, len(items)))()
        self._keep = []
        self.outputs = []
        for q, it in enumerate(items):
            kp, out = _fill_item(arr[q], it)
            self._keep += kp
            self.outputs.append(out)
        self._n = len(items)
        self._h = ctypes.c_void_p()
        _lib.check(self._lib.tsqr_batch_plan_create(arr, len(items), chain_tiles, arity, ctypes.byref(self._h)),
                   "tsqr_batch_plan_create")

    def run(self, stream=None):
        _lib.check(self._lib.tsqr_batch_plan_run(self._h, _stream(stream)), "tsqr_batch_plan_run")
        return self.outputs

    def results(self):
        """(status list, [(refinement steps, last ||dX||/||X||)]) of the last run (waits for it)."""
        st = (ctypes.c_int32 * self._n)()
        inf = (ctypes.c_double * (2 * self._n))()
        _lib.check(self._lib.tsqr_batch_plan_results(self._h, st, inf), "tsqr_batch_plan_results")
        return [st[q] for q in range(self._n)], [(int(inf[2 * q]), inf[2 * q + 1]) for q in range(self._n)]

    def close(self):
        if self._h:
            _lib.check(self._lib.tsqr_batch_plan_destroy(self._h), "tsqr_batch_plan_destroy")
            self._h = ctypes.c_void_p()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class Server:
    """Continuous-batching least-squares server on the current CUDA device.

    submit() queues one request (a dict as for batch_solve) and returns its ticket and
    its (R, X) output tensors, which are valid once poll() has returned the ticket.
    Requests still in flight are kept alive here until then. The worker is native (a C++
    thread inside the library); this class only marshals arguments.
    """

    def __init__(self, max_bytes: int = 0, max_batch: int = 256, streams: int = 2, chain_tiles: int = 0,
                 ctas_per_sm: int = 0, resident: bool = False, idle_us: int = 2000):
        """``resident``: admit requests into one persistent kernel that stays on the GPU
        (tsqr_server_create_resident; ``max_bytes`` is then its arena, ``idle_us`` how long
        it polls for work before it ends) instead of launching a batch per free stream."""
        self._lib = _lib.load()
        self._h = ctypes.c_void_p()
        self.resident = bool(resident)
        if resident:
            _lib.check(self._lib.tsqr_server_create_resident(max_bytes, chain_tiles, ctas_per_sm, idle_us,
                                                             ctypes.byref(self._h)), "tsqr_server_create_resident")
        else:
            _lib.check(self._lib.tsqr_server_create(max_bytes, max_batch, streams, chain_tiles, ctas_per_sm,
                                                    ctypes.byref(self._h)), "tsqr_server_create")
        self._live = {}

    def submit(self, item):
        slot = _lib.BatchItem()
        keep, out = _fill_item(slot, item)
        t = ctypes.c_int64(0)
        _lib.check(self._lib.tsqr_server_submit(self._h, ctypes.byref(slot), ctypes.byref(t)), "tsqr_server_submit")
        self._live[t.value] = keep
        return t.value, out

    def poll(self, max_count: int = 4096):
        """Completed requests as a list of (ticket, latency seconds, status)."""
        tk = (ctypes.c_int64 * max_count)()
        lat = (ctypes.c_double * max_count)()
        st = (ctypes.c_int32 * max_count)()
        c = ctypes.c_int32(0)
        _lib.check(self._lib.tsqr_server_poll(self._h, max_count, tk, lat, st, ctypes.byref(c)), "tsqr_server_poll")
        res = [(tk[i], lat[i], st[i]) for i in range(c.value)]
        for t, _, _ in res:
            self._live.pop(t, None)
        return res

    def drain(self):
        _lib.check(self._lib.tsqr_server_drain(self._h), "tsqr_server_drain")

    def stats(self):
        out = (ctypes.c_int64 * 6)()
        _lib.check(self._lib.tsqr_server_stats(self._h, out), "tsqr_server_stats")
        keys = (("submitted", "completed", "launches", "max_in_flight", "arena_bytes", "bytes_in_flight")
                if self.resident else
                ("submitted", "completed", "batches", "max_batch", "budget_bytes", "bytes_in_flight"))
        return dict(zip(keys, list(out)))

    def close(self):
        if self._h:
            _lib.check(self._lib.tsqr_server_destroy(self._h), "tsqr_server_destroy")
            self._h = ctypes.c_void_p()
            self._live.clear()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def probe_fp64_peak(stream=None, clock: bool = False):
    """Measured burst FP64 FMA throughput of the current device in TFLOP/s (with
    ``clock``, also the SM clock in MHz the probe ran at)."""
    lib = _lib.load()
    out = ctypes.c_double(0.0)
    mhz = ctypes.c_double(0.0)
    _lib.check(lib.tsqr_probe_fp64_peak(_stream(stream), ctypes.byref(out), ctypes.byref(mhz)),
               "tsqr_probe_fp64_peak")
    return (out.value, mhz.value) if clock else out.value


def _check_host(t, name, rows=None, cols=None):
    import torch
    if not isinstance(t, torch.Tensor) or t.is_cuda or t.dtype != torch.float64 or t.dim() != 2:
        raise TypeError(f"{name} must be a 2-D float64 CPU tensor")
    if t.stride(0) != 1:
        raise ValueError(f"{name} must be column-major (stride(0) == 1); use colmajor()")
    if rows is not None and t.shape[0] != rows:
        raise ValueError(f"{name} has {t.shape[0]} rows, expected {rows}")
    if cols is not None and t.shape[1] != cols:
        raise ValueError(f"{name} has {t.shape[1]} columns, expected {cols}")
    return max(t.stride(1), max(1, t.shape[0]))


def qr_solve_host(A, B=None, Q=None, R=None, X=None, leaf_h: int = 256, arity: int = 2, two_level: bool = True,
                  cluster: bool = False, stream=None, after=None, done=None, status=None):
    """The whole FP64 path on host (CPU) tensors through tsqr_qr_solve_host: copies A (and
    B) in, factors, forms the thin Q, R and X = R^{-1} (Q^T B)[0:n], copies them back into
    the given column-major float64 CPU tensors (pinned ones make every copy asynchronous;
    the outputs are valid once the stream reaches the call's end). ``after`` / ``done``:
    optional torch.cuda.Event the call's kernels wait for / that is recorded after them.
    ``status``: optional pinned int32 CPU tensor receiving 4 for a singular R."""
    lib = _lib.load()
    lda = _check_host(A, "A")
    m, n = A.shape
    ldb = _check_host(B, "B", rows=m) if B is not None else m
    k = B.shape[1] if B is not None else 0
    ldx = _check_host(X, "X", rows=n, cols=k) if X is not None else n
    ldq = _check_host(Q, "Q", rows=m, cols=n) if Q is not None else m
    ldr = _check_host(R, "R", rows=n, cols=n) if R is not None else n
    flags = (TWO_LEVEL if two_level else 0) | (CLUSTER if cluster else 0)
    ptr = (lambda t: t.data_ptr() if t is not None else None)
    ev = (lambda e: ctypes.c_void_p(e.cuda_event) if e is not None else None)
    _lib.check(lib.tsqr_qr_solve_host(A.data_ptr(), m, n, lda, ptr(B), ldb, k, ptr(Q), ldq, ptr(R), ldr, ptr(X), ldx,
                                      ptr(status), leaf_h, arity, flags, _stream(stream), ev(after), ev(done)),
               "tsqr_qr_solve_host")
    return Q, R, X


def set_mixed_wy_min_n(min_n: int) -> int:
    """Mixed-precision items with at least ``min_n`` columns factor their FP32 leaf chains
    by compact-WY panels with 3xTF32 tensor-core updates (0: never). Returns the previous
    threshold (tsqr_set_mixed_wy_min_n)."""
    return _lib.load().tsqr_set_mixed_wy_min_n(int(min_n))


def set_apply_tile_pairs(on: bool) -> bool:
    """Q^T b / Q b with one column: tile pairs per warp (True, the default) or one warp per
    tile in sequence (False). Returns the previous setting (tsqr_set_apply_tile_pairs)."""
    return bool(_lib.load().tsqr_set_apply_tile_pairs(1 if on else 0))


def error_word(stream=None) -> int:
    """Reads and clears the device error word (tsqr_error_word; waits for the stream):
    bit 1 = a bounded device wait gave up, bit 2 = an index check of a TSQR_CHECK build."""
    w = ctypes.c_int32(0)
    st = _lib.load().tsqr_error_word(_stream(stream), ctypes.byref(w))
    if st not in (0, 5):
        _lib.check(st, "tsqr_error_word")
    return w.value


def probe_dmma_peak(stream=None, clock: bool = False):
    """Measured burst FP64 tensor-core (DMMA) throughput in TFLOP/s (with ``clock``, also
    the SM clock in MHz), for comparison with probe_fp64_peak."""
    lib = _lib.load()
    out = ctypes.c_double(0.0)
    mhz = ctypes.c_double(0.0)
    _lib.check(lib.tsqr_probe_dmma_peak(_stream(stream), ctypes.byref(out), ctypes.byref(mhz)),
               "tsqr_probe_dmma_peak")
    return (out.value, mhz.value) if clock else out.value


def profile_collect(fn):
    """Runs fn() with launch profiling on and returns (fn's result, [(class, ms), ...])."""
    lib = _lib.load()
    _lib.check(lib.tsqr_profile_start(), "tsqr_profile_start")
    try:
        out = fn()
    finally:
        cap = 1 << 16
        kinds = (ctypes.c_int32 * cap)()
        ms = (ctypes.c_float * cap)()
        cnt = ctypes.c_int64(0)
        st = lib.tsqr_profile_stop(cap, kinds, ms, ctypes.byref(cnt))
    _lib.check(st, "tsqr_profile_stop")
    n = min(cnt.value, cap)
    return out, [(PROFILE_KINDS.get(kinds[i], str(kinds[i])), ms[i]) for i in range(n)]


def plan_describe(m, n, leaf_h, arity=2, two_level=True, nc=None, sms=None):
    """Host-only plan summary for the current device (or a device with `sms` SMs and
    GB300 shared-memory sizes)."""
    import torch
    lib = _lib.load()
    if sms is None and torch.cuda.is_available():
        p = torch.cuda.get_device_properties(torch.cuda.current_device())
        sms = p.multi_processor_count
    sms = sms or 152
    out = (ctypes.c_int64 * 8)()
    st = lib.tsqr_plan_describe(m, n, nc or n, leaf_h, arity, TWO_LEVEL if two_level else 0, sms, 233472,
                                1024, 232448, out, None, 0, None, 0)
    _lib.check(st, "tsqr_plan_describe")
    keys = ["m", "n", "leaves", "tile_rows", "jobs", "tiles", "launches", "ctas_per_sm"]
    return dict(zip(keys, list(out)))


def lstsq(A, B, leaf_h: int = 256, arity: int = 2, two_level: bool = True, prec: int = FP64,
          max_refine: int = 10, X=None, stream=None, info: bool = False, cluster: bool = False):
    """X = argmin ||A X - B|| for column-major float64 CUDA tensors (A m-by-n, B m-by-k).

    prec FP64: TSQR of [A | B] with Q^T B fused, then back substitution. MIXED: FP32
    leaves, FP64 tree, FP64 iterative refinement. With ``info`` also returns the list of
    ||dX||/||X|| per refinement step.
    """
    import torch
    lib = _lib.load()
    lda = _check_mat(A, "A")
    m, n = A.shape
    ldb = _check_mat(B, "B", rows=m)
    k = B.shape[1]
    if X is None:
        X = torch.empty((k, n), dtype=torch.float64, device=A.device).t()
    ldx = _check_mat(X, "X", rows=n, cols=k)
    hist = (ctypes.c_double * (max_refine + 1))()
    flags = (TWO_LEVEL if two_level else 0) | (CLUSTER if cluster else 0)
    st = lib.tsqr_lstsq(A.data_ptr(), m, n, lda, B.data_ptr(), ldb, k, X.data_ptr(), ldx, leaf_h, arity,
                        prec, flags, max_refine, _stream(stream), hist if info else None)
    _lib.check(st, "tsqr_lstsq")
    if info:
        return X, list(hist)
    return X
